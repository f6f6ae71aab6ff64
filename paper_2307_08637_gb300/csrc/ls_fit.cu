// ls_fit.cu -- the "training" side of learned SampleSort on GB300:
//   Sample(A, l, r) of Alg. 2-5 (counter-based SplitMix64 positions),
//   segmented sample sort (bitonic chunks + merge path),
//   the FP64 closed-form least-squares fit of the two-layer RMI (Sec. 2.1-2.2),
//   the monotone clamps of Sec. 4,
//   the exact learned pivots (Alg. 4's implicit pivots, as lower bounds),
//   Alg. 5's model choice, SampleSort splitter tables with IPS4o equality
//   buckets (Sec. 2.4), the radix directory over a pivot table, and the
//   forward / backward pass of the fit objective.
#include <cfloat>
#include <cmath>

#include "ls_kernels.h"

namespace lsg {

namespace {

constexpr int kTPB = 256;

inline unsigned grid_for(uint64_t n, int tpb = kTPB) { return (unsigned)((n + tpb - 1) / tpb); }

// Largest f in [0, n) with prefix[f] <= g (prefix has n+1 non-decreasing entries).
__device__ __forceinline__ uint32_t find_seg(const uint64_t* __restrict__ prefix, uint32_t n, uint64_t g) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (prefix[mid] <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Closed-form least squares y = a X + b from (n, sum X, sum y, sum Xy, sum X^2),
// slope clamped at 0 (every model non-decreasing).
__device__ __forceinline__ void linfit(double n, double sx, double sy, double sxy, double sxx, double* a,
                                       double* b) {
  double t1 = __dmul_rn(n, sxx);
  double t2 = __dmul_rn(sx, sx);
  double D = __dsub_rn(t1, t2);
  double A = 0.0;
  if (D > 0.0) {
    double u1 = __dmul_rn(n, sxy);
    double u2 = __dmul_rn(sx, sy);
    double num = __dsub_rn(u1, u2);
    A = __ddiv_rn(num, D);
  }
  A = dmax(A, 0.0);
  double ax = __dmul_rn(A, sx);
  double r = __dsub_rn(sy, ax);
  *a = A;
  *b = __ddiv_rn(r, n);
}

// The same four sums over one chunk [j0, j1) (at most kChunk = 256
// positions) by a whole warp, as a fixed pairwise tree: lane l forms the
// terms of positions j0 + 8l .. j0 + 8l + 7 (+0.0 beyond j1), adds them in
// pairs, and the lanes combine in pairs (lane 2k takes lane 2k+1's partial,
// then 4k takes 4k+2's, ...), so lane 0 ends with the complete binary tree
// over the 256 positions.  Every term is >= +0 (X >= 0 because x0 is the
// smallest key of the range; y, X y, X X >= 0), so the zero padding changes
// no addition: this is the tree that halves the list pair by pair and
// carries an odd last value.  Result valid in lane 0.
__device__ __forceinline__ void warp_chunk_sums(const uint64_t* __restrict__ s, uint64_t j0, uint64_t j1, double x0,
                                                double Sd, int dt, double out[4]) {
  const unsigned lane = threadIdx.x & 31;
  double t[4][8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const uint64_t j = j0 + 8 * lane + e;
    if (j < j1) {
      const double X = __dsub_rn(ord_value(s[j], dt), x0);
      const double y = __ddiv_rn(__ull2double_rn(j), Sd);
      t[0][e] = X;
      t[1][e] = y;
      t[2][e] = __dmul_rn(X, y);
      t[3][e] = __dmul_rn(X, X);
    } else {
      t[0][e] = t[1][e] = t[2][e] = t[3][e] = 0.0;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double v = __dadd_rn(__dadd_rn(__dadd_rn(t[q][0], t[q][1]), __dadd_rn(t[q][2], t[q][3])),
                         __dadd_rn(__dadd_rn(t[q][4], t[q][5]), __dadd_rn(t[q][6], t[q][7])));
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) v = __dadd_rn(v, __shfl_down_sync(0xFFFFFFFFu, v, d));
    out[q] = v;
  }
}

// Fixed pairwise tree over m partials, done by one thread in place:
// p[i] = p[2i] + p[2i+1], an odd last value carried up (same shape as the
// oracle's tree_sum).  Empty -> +0.0.
__device__ double thread_tree_sum(double* p, uint64_t m) {
  if (m == 0) return 0.0;
  while (m > 1) {
    uint64_t h = m >> 1;
    for (uint64_t i = 0; i < h; ++i) p[i] = __dadd_rn(p[2 * i], p[2 * i + 1]);
    if (m & 1) p[h] = p[m - 1];
    m = h + (m & 1);
  }
  return p[0];
}

// thread_tree_sum's tree done by a warp, in place, over K arrays at once
// (p[q] + q * stride, m partials each): every level adds the pairs
// (2i, 2i+1) with 32 lanes at a time (all reads of a group before its
// writes; later groups read only indices above the ones written) and
// carries an odd last value, so each total is bit-identical.  Every lane
// returns the totals.
template <int K>
__device__ void warp_tree_sum_inplace(double* p, uint64_t stride, uint64_t m, double (&out)[K]) {
  const unsigned lane = threadIdx.x & 31;
  if (m == 0) {
#pragma unroll
    for (int q = 0; q < K; ++q) out[q] = 0.0;
    return;
  }
  while (m > 1) {
    const uint64_t h = m >> 1;
    for (uint64_t i0 = 0; i0 < h; i0 += 32) {
      const uint64_t i = i0 + lane;
      double v[K];
#pragma unroll
      for (int q = 0; q < K; ++q) v[q] = i < h ? __dadd_rn(p[q * stride + 2 * i], p[q * stride + 2 * i + 1]) : 0.0;
      __syncwarp();
      if (i < h)
#pragma unroll
        for (int q = 0; q < K; ++q) p[q * stride + i] = v[q];
      __syncwarp();
    }
    if ((m & 1) && lane == 0)
#pragma unroll
      for (int q = 0; q < K; ++q) p[q * stride + h] = p[q * stride + m - 1];
    __syncwarp();
    m = h + (m & 1);
  }
#pragma unroll
  for (int q = 0; q < K; ++q) out[q] = p[q * stride];
}

// The same tree done by a block over K arrays staged in shared memory
// (s: K * m words, filled from p[q] + q * stride), in place: each level's
// reads happen before its writes (a barrier between them).  Every thread
// returns the totals.
template <int K>
__device__ void block_tree_sum_smem(const double* p, uint64_t stride, uint32_t m, double* s, double (&out)[K]) {
  for (uint32_t i = threadIdx.x; i < m; i += blockDim.x)
#pragma unroll
    for (int q = 0; q < K; ++q) s[q * m + i] = p[q * stride + i];
  __syncthreads();
  uint32_t cur = m;
  while (cur > 1) {
    const uint32_t h = cur >> 1;
    constexpr int kPer = 4;  // pairs per thread per round (h <= 4 * blockDim.x per round)
    for (uint32_t i0 = 0; i0 < h; i0 += kPer * blockDim.x) {
      double v[kPer][K];
#pragma unroll
      for (int r = 0; r < kPer; ++r) {
        const uint32_t i = i0 + r * blockDim.x + threadIdx.x;
#pragma unroll
        for (int q = 0; q < K; ++q) v[r][q] = i < h ? __dadd_rn(s[q * m + 2 * i], s[q * m + 2 * i + 1]) : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < kPer; ++r) {
        const uint32_t i = i0 + r * blockDim.x + threadIdx.x;
        if (i < h)
#pragma unroll
          for (int q = 0; q < K; ++q) s[q * m + i] = v[r][q];
      }
      __syncthreads();
    }
    if ((cur & 1) && threadIdx.x == 0)
#pragma unroll
      for (int q = 0; q < K; ++q) s[q * m + h] = s[q * m + cur - 1];
    __syncthreads();
    cur = h + (cur & 1);
  }
#pragma unroll
  for (int q = 0; q < K; ++q) out[q] = s[q * m];
  __syncthreads();
}

// Same tree done by a whole block, ping-ponging between p and q (same size).
__device__ double block_tree_sum(double* p, double* q, uint64_t m) {
  if (m == 0) return 0.0;
  while (m > 1) {
    uint64_t h = m >> 1;
    for (uint64_t i = threadIdx.x; i < h; i += blockDim.x) q[i] = __dadd_rn(p[2 * i], p[2 * i + 1]);
    if ((m & 1) && threadIdx.x == 0) q[h] = p[m - 1];
    __syncthreads();
    double* t = p;
    p = q;
    q = t;
    m = h + (m & 1);
  }
  double r = p[0];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------ sampling

__global__ void k_sample_gather(FreshArgs f, RunParams rp, uint64_t* __restrict__ samp) {
  pdl_wait();
  uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (g >= f.total_samples) return;
  uint32_t fi = find_seg(f.samp_prefix, f.nfresh, g);
  uint64_t j = g - f.samp_prefix[fi];
  uint32_t pi = f.fresh[fi];
  const Item& it = f.items[pi];
  const Plan& pl = f.plans[pi];
  uint64_t n = it.n;
  uint64_t pos;
  if ((uint64_t)pl.S >= n) {
    pos = j;  // S == n: every key, in index order
  } else {
    uint64_t h = seed_item(rp.seed, it.segment, it.level, it.gidx);
    uint64_t r = splitmix64(h + (j + 1) * kGolden);
    pos = __umul64hi(r, n);
  }
  const uint64_t* src = it.buf ? f.keysB : f.keysA;
  samp[pl.sample_off + j] = ord_of(src[it.lo + pos], rp.dt);
}

// Sample(A) of Alg. 2-5 for one array with a caller-given stream seed h:
// key j of the sample is A[floor(u_j n / 2^64)], u_j = SplitMix64 output at
// h + (j+1) * golden gamma (with replacement); S >= n takes A in order.
__global__ void k_sample_keys(const uint64_t* __restrict__ keys, uint64_t n, uint64_t S, uint64_t h,
                              uint64_t* __restrict__ out) {
  pdl_wait();
  uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (j >= S) return;
  uint64_t pos = j;
  if (S < n) pos = __umul64hi(splitmix64(h + (j + 1) * kGolden), n);
  out[j] = keys[pos];
}

__global__ void k_dups(FreshArgs f, const uint64_t* __restrict__ samp) {
  pdl_wait();
  uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  bool valid = g < f.total_samples;
  uint32_t fi = valid ? find_seg(f.samp_prefix, f.nfresh, g) : 0xFFFFFFFFu;
  bool dup = false;
  if (valid) {
    uint64_t j = g - f.samp_prefix[fi];
    dup = (j > 0) && (samp[g] == samp[g - 1]);
  }
  unsigned dmask = __ballot_sync(0xFFFFFFFFu, dup);
  unsigned peers = __match_any_sync(0xFFFFFFFFu, fi);
  unsigned lane = threadIdx.x & 31;
  if (valid && lane == (unsigned)(__ffs(peers) - 1)) {
    unsigned c = __popc(dmask & peers);
    if (c) atomicAdd(&f.plans[f.fresh[fi]].dups, (unsigned long long)c);
  }
}

// ------------------------------------------------ segmented sample sort

constexpr int kSortTPB = 1024;  // threads of a chunk sort: two of the chunk's 2048 keys each
static_assert(kSortChunk == 2 * kSortTPB, "two keys per thread");

// Bitonic sort of one chunk of kSortChunk keys (padding ~0).  Each warp
// holds 64 consecutive keys, two per lane: the stages whose pairs lie inside
// 64 keys run in registers (lane shuffles), the wider ones in shared memory
// with one thread per pair.
__global__ void __launch_bounds__(kSortTPB) k_sort_chunks(uint64_t* __restrict__ a, const uint64_t* __restrict__ off,
                                                      const uint64_t* __restrict__ cpre, uint32_t nseg) {
  pdl_wait();
  __shared__ uint64_t sm[kSortChunk];
  uint64_t c = blockIdx.x;
  uint32_t s = find_seg(cpre, nseg, c);
  uint64_t base = off[s] + (c - cpre[s]) * kSortChunk;
  uint64_t end = off[s + 1];
  if (end > base + kSortChunk) end = base + kSortChunk;
  uint32_t len = (uint32_t)(end - base);
  for (uint32_t i = threadIdx.x; i < kSortChunk; i += blockDim.x) sm[i] = (i < len) ? a[base + i] : ~0ull;
  __syncthreads();
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t e0 = 64 * wid + 2 * lane;  // this lane's keys: e0 and e0 + 1
  uint64_t r0 = sm[e0], r1 = sm[e0 + 1];
  // stages j = jtop .. 1 of the bitonic merge of size k, in registers
  auto reg_stages = [&](uint32_t k, uint32_t jtop) {
    const bool up = (e0 & k) == 0;  // k >= 2: e0 and e0 + 1 agree on bit k
    for (uint32_t j = jtop; j >= 2; j >>= 1) {
      const uint64_t y0 = __shfl_xor_sync(0xFFFFFFFFu, r0, j >> 1);
      const uint64_t y1 = __shfl_xor_sync(0xFFFFFFFFu, r1, j >> 1);
      const bool keep_min = ((e0 & j) == 0) == up;
      r0 = keep_min ? (r0 < y0 ? r0 : y0) : (r0 < y0 ? y0 : r0);
      r1 = keep_min ? (r1 < y1 ? r1 : y1) : (r1 < y1 ? y1 : r1);
    }
    const uint64_t mn = r0 < r1 ? r0 : r1, mx = r0 < r1 ? r1 : r0;
    r0 = up ? mn : mx;
    r1 = up ? mx : mn;
  };
  for (uint32_t k = 2; k <= 64; k <<= 1) reg_stages(k, k >> 1);
  for (uint32_t k = 128; k <= kSortChunk; k <<= 1) {
    sm[e0] = r0;
    sm[e0 + 1] = r1;
    __syncthreads();
    for (uint32_t j = k >> 1; j >= 64; j >>= 1) {
      const uint32_t p = threadIdx.x;
      const uint32_t i = ((p & ~(j - 1)) << 1) | (p & (j - 1));
      const uint64_t x = sm[i], y = sm[i + j];
      if ((x > y) == ((i & k) == 0)) {
        sm[i] = y;
        sm[i + j] = x;
      }
      __syncthreads();
    }
    r0 = sm[e0];
    r1 = sm[e0 + 1];
    reg_stages(k, 32);
  }
  sm[e0] = r0;
  sm[e0 + 1] = r1;
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) a[base + i] = sm[i];
}

// Merge-path split of diagonal d between sorted runs A (na keys) and B (nb
// keys): the number of A's keys among the first d outputs (ties take A).
// One warp, 32 probes per round, so a search of 2^20 positions takes four
// rounds of loads instead of twenty dependent ones.  Every lane returns it.
__device__ __forceinline__ uint64_t warp_merge_split(const uint64_t* __restrict__ A, uint64_t na,
                                                     const uint64_t* __restrict__ B, uint64_t nb, uint64_t d) {
  const unsigned lane = threadIdx.x & 31;
  uint64_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
  while (lo < hi) {  // uniform across the warp
    const uint64_t step = (hi - lo + 31) / 32;
    const uint64_t i = lo + lane * step;
    const bool in = i < hi;
    const bool p = in && A[i] <= B[d - 1 - i];  // the split lies above i
    const unsigned mp = __ballot_sync(0xFFFFFFFFu, p), mf = __ballot_sync(0xFFFFFFFFu, in && !p);
    const uint64_t nlo = mp ? lo + (uint64_t)(31 - __clz(mp)) * step + 1 : lo;
    const uint64_t nhi = mf ? lo + (uint64_t)(__ffs(mf) - 1) * step : hi;
    lo = nlo;
    hi = nhi;
  }
  return lo;
}

// One merge pass: within each segment, runs [2pw, 2pw+w) and [2pw+w, 2pw+2w)
// are merged (merge path, ties take the left run).  A block produces one
// chunk of kSortChunk outputs (a chunk lies inside one pair of runs): two
// warps find the splits at the chunk's ends, the block stages the two input
// slices in shared memory, and each thread merges eight outputs from there.
constexpr int kMergeTPB = kSortChunk / 8;
__global__ void __launch_bounds__(kMergeTPB) k_merge_pass(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                          const uint64_t* __restrict__ off,
                                                          const uint64_t* __restrict__ cpre, uint32_t nseg,
                                                          uint64_t w) {
  pdl_wait();
  __shared__ uint64_t sm[kSortChunk];
  __shared__ uint64_t s_split[2];
  const uint64_t c = blockIdx.x;
  const uint32_t s = find_seg(cpre, nseg, c);
  const uint64_t sb = off[s];
  const uint64_t len = off[s + 1] - sb;
  const uint64_t o0 = (c - cpre[s]) * kSortChunk;
  if (o0 >= len) return;  // uniform across the block
  const uint64_t a0 = (o0 / (2 * w)) * (2 * w);
  const uint64_t a1 = a0 + w < len ? a0 + w : len;
  const uint64_t b1 = a0 + 2 * w < len ? a0 + 2 * w : len;
  const uint64_t na = a1 - a0, nbb = b1 - a1;
  const uint64_t* A = in + sb + a0;
  const uint64_t* Bv = in + sb + a1;
  const uint64_t d0 = o0 - a0;
  const uint64_t d1 = d0 + kSortChunk < na + nbb ? d0 + kSortChunk : na + nbb;
  const unsigned wid = threadIdx.x >> 5;
  if (wid < 2) {
    const uint64_t sp = warp_merge_split(A, na, Bv, nbb, wid ? d1 : d0);
    if ((threadIdx.x & 31) == 0) s_split[wid] = sp;
  }
  __syncthreads();
  const uint64_t i0 = s_split[0], i1 = s_split[1];
  const uint64_t j0 = d0 - i0, j1 = d1 - i1;
  const uint32_t la = (uint32_t)(i1 - i0), lb = (uint32_t)(j1 - j0);  // la + lb = d1 - d0 <= kSortChunk
  for (uint32_t t = threadIdx.x; t < la + lb; t += blockDim.x) sm[t] = t < la ? A[i0 + t] : Bv[j0 + t - la];
  __syncthreads();
  const uint64_t* SA = sm;
  const uint64_t* SB = sm + la;
  const uint32_t dt = 8 * threadIdx.x;
  if (dt >= la + lb) return;
  uint32_t lo = dt > lb ? dt - lb : 0, hi = dt < la ? dt : la;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (SA[mid] <= SB[dt - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  uint32_t i = lo, j = dt - lo;
  const uint32_t lim = la + lb - dt < 8 ? la + lb - dt : 8;
  uint64_t* o = out + sb + a0 + d0 + dt;
  for (uint32_t k = 0; k < lim; ++k) {
    const bool takeA = (j >= lb) || (i < la && SA[i] <= SB[j]);
    o[k] = takeA ? SA[i++] : SB[j++];
  }
}

// ---------------------------------------------------------------- fit

// Root partials staged in shared memory by the finish kernel (4 sums of
// up to this many chunks: 128 KB); more chunks take the global tree.
constexpr uint32_t kRootSmemChunks = 4096;

// One warp per root chunk of every candidate.
__global__ void k_fit_root_partials(FitArgs a, RunParams rp) {
  pdl_wait();
  const uint64_t g = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  if (g >= a.total_rchunks) return;  // uniform across the warp
  const uint32_t c = find_seg(a.rchunk_prefix, a.ncand, g);
  const uint64_t k = g - a.rchunk_prefix[c];
  const Plan& pl = a.plans[a.cand[c]];
  const uint64_t S = pl.S;
  const uint64_t* s = a.samp + pl.sample_off;
  const double x0 = ord_value(s[0], rp.dt);
  const uint64_t j0 = k * kChunk;
  const uint64_t j1 = j0 + kChunk < S ? j0 + kChunk : S;
  double out[4];
  warp_chunk_sums(s, j0, j1, x0, __ull2double_rn(S), rp.dt, out);
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 4; ++q) a.rpart[q * a.total_rchunks + g] = out[q];
}

// Per candidate: tree-combine the root chunk partials, fit the root.
__global__ void k_fit_root_finish(FitArgs a, RunParams rp) {
  pdl_wait();
  uint32_t c = blockIdx.x;
  const Plan& pl = a.plans[a.cand[c]];
  uint64_t b0 = a.rchunk_prefix[c];
  uint64_t m = a.rchunk_prefix[c + 1] - b0;
  __shared__ double sums[4];
  if (m <= kRootSmemChunks) {  // the candidate's partials fit in shared memory
    extern __shared__ double s_part[];
    double out[4];
    block_tree_sum_smem<4>(a.rpart + b0, a.total_rchunks, (uint32_t)m, s_part, out);
    if (threadIdx.x == 0)
      for (int q = 0; q < 4; ++q) sums[q] = out[q];
  } else {
    for (int q = 0; q < 4; ++q) {
      double* p = a.rpart + q * a.total_rchunks + b0;
      double* t = a.rpart + (4 + q) * a.total_rchunks + b0;  // ping-pong half
      double v = block_tree_sum(p, t, m);
      if (threadIdx.x == 0) sums[q] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t S = pl.S;
    const uint64_t* s = a.samp + pl.sample_off;
    DModel& m0 = a.models[pl.model];
    m0.xmin = ord_value(s[0], rp.dt);
    m0.xmax = ord_value(s[S - 1], rp.dt);
    m0.rx0 = m0.xmin;
    double ra, rb;
    linfit(__ull2double_rn(S), sums[0], sums[1], sums[2], sums[3], &ra, &rb);
    m0.ra = ra;
    m0.rb = rb;
    m0.L = a.L;
    m0.S = (uint32_t)S;
    m0.leaf_off = (uint64_t)pl.model * a.L;
    m0.ok = 0;
  }
}

// Route every sample point to its leaf (stored), then mark run starts.
__global__ void k_fit_route_leaf(FitArgs a, RunParams rp, uint32_t* __restrict__ leaf_of) {
  pdl_wait();
  uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (g >= a.total_cand_samples) return;
  uint32_t c = find_seg(a.cand_soff, a.ncand, g);
  uint64_t j = g - a.cand_soff[c];
  const Plan& pl = a.plans[a.cand[c]];
  DModel m = a.models[pl.model];
  leaf_of[g] = root_leaf(m, ord_value(a.samp[pl.sample_off + j], rp.dt));
}

__global__ void k_fit_route_starts(FitArgs a, const uint32_t* __restrict__ leaf_of) {
  pdl_wait();
  uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (g >= a.total_cand_samples) return;
  uint32_t c = find_seg(a.cand_soff, a.ncand, g);
  uint64_t j = g - a.cand_soff[c];
  uint64_t S = a.cand_soff[c + 1] - a.cand_soff[c];
  uint32_t* ls = a.leaf_start + (uint64_t)c * (a.L + 1);
  uint32_t lf = leaf_of[g];
  lf = lf < a.L ? lf : a.L - 1;  // root_leaf is already clamped; never index past the run table
  if (j == 0) {
    for (uint32_t i = 0; i <= lf; ++i) ls[i] = 0;
  } else {
    uint32_t prev = leaf_of[g - 1];
    prev = prev < a.L ? prev : a.L - 1;
    for (uint32_t i = prev + 1; i <= lf; ++i) ls[i] = (uint32_t)j;
  }
  if (j == S - 1) {
    for (uint32_t i = lf + 1; i <= a.L; ++i) ls[i] = (uint32_t)S;
  }
}

// Leaves of at most kLaneLeafMax samples (one chunk) are fitted by one lane
// each (k_fit_leaf_lane) instead of a warp per chunk and a warp per leaf:
// with few samples per leaf (retrained models of small buckets) the
// warp-wide trees cost per leaf, not per sample, on a slow FP64 pipe.
constexpr uint64_t kLaneLeafMax = 32;

__global__ void k_fit_leaf_chunk_count(FitArgs a) {
  pdl_wait();
  uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  uint64_t tot = (uint64_t)a.ncand * a.L;
  if (g > tot) return;
  if (g == tot) {
    a.lchunk_cnt[g] = 0;
    return;
  }
  uint32_t c = (uint32_t)(g / a.L), i = (uint32_t)(g % a.L);
  const uint32_t* ls = a.leaf_start + (uint64_t)c * (a.L + 1);
  uint64_t cnt = ls[i + 1] > ls[i] ? ls[i + 1] - ls[i] : 0;
  a.lchunk_cnt[g] = cnt <= kLaneLeafMax ? 0 : (cnt + kChunk - 1) / kChunk;  // short leaves: k_fit_leaf_lane
}

// One warp per leaf chunk of every candidate.
__global__ void k_fit_leaf_partials(FitArgs a, RunParams rp) {
  pdl_wait();
  const uint64_t g = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint32_t tot = a.ncand * a.L;
  if (g >= a.lchunk_prefix[tot] || g >= a.lchunk_bound) return;  // uniform across the warp
  const uint32_t ci = find_seg(a.lchunk_prefix, tot, g);
  const uint64_t k = g - a.lchunk_prefix[ci];
  const uint32_t c = ci / a.L, i = ci % a.L;
  const Plan& pl = a.plans[a.cand[c]];
  const uint64_t* s = a.samp + pl.sample_off;
  const uint32_t* ls = a.leaf_start + (uint64_t)c * (a.L + 1);
  const uint64_t S = pl.S;
  const uint64_t en = ls[i + 1] < S ? ls[i + 1] : S;
  const uint64_t st = ls[i] < en ? ls[i] : en;
  if (st >= en) return;
  const double x0 = ord_value(s[st], rp.dt);
  const uint64_t j0 = st + k * kChunk;
  const uint64_t j1 = j0 + kChunk < en ? j0 + kChunk : en;
  double out[4];
  warp_chunk_sums(s, j0, j1, x0, __ull2double_rn((uint64_t)pl.S), rp.dt, out);
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 4; ++q) a.lpart[q * a.lchunk_bound + g] = out[q];
}

// thread_tree_sum's tree over m <= 32 partials held one per lane (lane k:
// p[k]): every level adds the pairs (2i, 2i+1) and carries an odd last
// value, so the total is bit-identical.  Every lane returns it.
__device__ __forceinline__ double warp_tree_sum32(double v, uint32_t m, unsigned lane) {
  while (m > 1) {  // uniform
    const uint32_t h = m >> 1;
    const double x = __shfl_sync(0xFFFFFFFFu, v, (2 * lane) & 31);
    const double y = __shfl_sync(0xFFFFFFFFu, v, (2 * lane + 1) & 31);
    const double z = __shfl_sync(0xFFFFFFFFu, v, (m - 1) & 31);
    if (lane < h) v = __dadd_rn(x, y);
    else if ((m & 1) && lane == h) v = z;
    m = h + (m & 1);
  }
  return __shfl_sync(0xFFFFFFFFu, v, 0);
}

// One warp per (candidate, leaf): the leaf's four sums (a warp tree over its
// chunk partials), its least-squares line and raw clamps.
__global__ void k_fit_leaf_finish(FitArgs a, RunParams rp, uint32_t* __restrict__ leaf_cnt) {
  pdl_wait();
  const uint64_t g = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const unsigned lane = threadIdx.x & 31;
  if (g >= (uint64_t)a.ncand * a.L) return;  // uniform across the warp
  uint32_t c = (uint32_t)(g / a.L), i = (uint32_t)(g % a.L);
  const Plan& pl = a.plans[a.cand[c]];
  const uint64_t* s = a.samp + pl.sample_off;
  const uint32_t* ls = a.leaf_start + (uint64_t)c * (a.L + 1);
  uint64_t S = pl.S;
  uint64_t en = ls[i + 1] < S ? ls[i + 1] : S;
  uint64_t st = ls[i] < en ? ls[i] : en;
  uint64_t cnt = en - st;
  if (cnt != 0 && cnt <= kLaneLeafMax) return;  // k_fit_leaf_lane's leaf (uniform across the warp)
  const uint32_t leaf_off = a.models[pl.model].leaf_off;
  Leaf l;
  if (cnt == 0) {
    l.x0 = a.models[pl.model].xmin;
    l.a = 0.0;
    l.b = 0.0;
    l.lo = 0.0;
    l.hi = 0.0;
  } else {
    const uint64_t p0 = a.lchunk_prefix[g];
    const uint64_t nch = a.lchunk_prefix[g + 1] - p0;
    double sm[4];
    if (nch <= 32) {
      for (int q = 0; q < 4; ++q) {
        const double v = lane < nch ? a.lpart[q * a.lchunk_bound + p0 + lane] : 0.0;
        sm[q] = warp_tree_sum32(v, (uint32_t)nch, lane);
      }
    } else {
      warp_tree_sum_inplace<4>(a.lpart + p0, a.lchunk_bound, nch, sm);
    }
    if (lane == 0) {
      double x_first = ord_value(s[st], rp.dt);
      double x_last = ord_value(s[en - 1], rp.dt);
      l.x0 = x_first;
      linfit(__ull2double_rn(cnt), sm[0], sm[1], sm[2], sm[3], &l.a, &l.b);
      l.lo = leaf_eval(l, x_first);  // raw min of the leaf (slope >= 0)
      l.hi = leaf_eval(l, x_last);   // raw max
    }
  }
  if (lane == 0) {
    a.leaves[leaf_off + i] = l;
    leaf_cnt[leaf_off + i] = (uint32_t)cnt;
  }
}

// One lane per (candidate, leaf) of 1..kLaneLeafMax samples: the four sums
// as the same fixed pairwise tree as warp_chunk_sums (the complete binary
// tree over the chunk, zero padded; adding +0.0 to a term >= +0 is exact),
// built in sample order like a binary counter: a new term enters level 0,
// equal levels merge (earlier partial + later), and at the end the pending
// partials combine from the lowest level up, which is the padded tree's
// right spine.  Then the leaf's line and raw clamps as in k_fit_leaf_finish.
__global__ void k_fit_leaf_lane(FitArgs a, RunParams rp, uint32_t* __restrict__ leaf_cnt) {
  pdl_wait();
  constexpr int kLv = 6;  // levels of a 32-term tree
  static_assert(kLaneLeafMax <= (1u << (kLv - 1)), "the counter holds 2^(kLv-1) terms");
  const uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (g >= (uint64_t)a.ncand * a.L) return;
  const uint32_t c = (uint32_t)(g / a.L), i = (uint32_t)(g % a.L);
  const Plan& pl = a.plans[a.cand[c]];
  const uint64_t* s = a.samp + pl.sample_off;
  const uint32_t* ls = a.leaf_start + (uint64_t)c * (a.L + 1);
  const uint64_t S = pl.S;
  const uint64_t en = ls[i + 1] < S ? ls[i + 1] : S;
  const uint64_t st = ls[i] < en ? ls[i] : en;
  const uint64_t cnt = en - st;
  if (cnt == 0 || cnt > kLaneLeafMax) return;
  const double x0 = ord_value(s[st], rp.dt), Sd = __ull2double_rn(S);
  double lv[4][kLv];
  uint32_t mask = 0;
  for (uint64_t j = st; j < en; ++j) {
    const double X = __dsub_rn(ord_value(s[j], rp.dt), x0);
    const double y = __ddiv_rn(__ull2double_rn(j), Sd);
    double cy[4] = {X, y, __dmul_rn(X, y), __dmul_rn(X, X)};
    bool open = true;
#pragma unroll
    for (int k = 0; k < kLv; ++k) {
      if (!open) continue;
      if (mask & (1u << k)) {
#pragma unroll
        for (int q = 0; q < 4; ++q) cy[q] = __dadd_rn(lv[q][k], cy[q]);
        mask &= ~(1u << k);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) lv[q][k] = cy[q];
        mask |= 1u << k;
        open = false;
      }
    }
  }
  double sm[4] = {0.0, 0.0, 0.0, 0.0};
  bool have = false;
#pragma unroll
  for (int k = 0; k < kLv; ++k) {
    if (!(mask & (1u << k))) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) sm[q] = have ? __dadd_rn(lv[q][k], sm[q]) : lv[q][k];
    have = true;
  }
  Leaf l;
  const double x_last = ord_value(s[en - 1], rp.dt);
  l.x0 = x0;
  linfit(__ull2double_rn(cnt), sm[0], sm[1], sm[2], sm[3], &l.a, &l.b);
  l.lo = leaf_eval(l, x0);  // raw min of the leaf (slope >= 0)
  l.hi = leaf_eval(l, x_last);  // raw max
  const uint32_t leaf_off = a.models[pl.model].leaf_off;
  a.leaves[leaf_off + i] = l;
  leaf_cnt[leaf_off + i] = (uint32_t)cnt;
}

// Monotone RMI (Sec. 4): hi_i = max(0, max over non-empty j <= i of raw
// maxima); lo_i = max(raw_lo_i, hi_{i-1}); empty leaves take hi_{i-1}.  The
// values are never -0.0 and never NaN for a finite model, so max is
// associative and a parallel prefix max gives the sequential result bit for
// bit.  One block per candidate; also sets the model's finite flag.
__global__ void __launch_bounds__(1024) k_fit_monotone(FitArgs a, const uint32_t* __restrict__ leaf_cnt) {
  pdl_wait();
  uint32_t c = blockIdx.x;
  const Plan& pl = a.plans[a.cand[c]];
  DModel& md = a.models[pl.model];
  Leaf* lv = a.leaves + md.leaf_off;
  const uint32_t* cn = leaf_cnt + md.leaf_off;
  uint32_t L = a.L;
  uint32_t per = (L + blockDim.x - 1) / blockDim.x;
  uint32_t i0 = threadIdx.x * per;
  double loc = 0.0;  // running max of raw maxima in my range (floor +0.0 is the initial hi)
  bool fin = true;
  for (uint32_t i = i0; i < i0 + per && i < L; ++i) {
    if (cn[i]) loc = dmax(loc, lv[i].hi);
    Leaf l = lv[i];
    fin = fin && isfinite(l.a) && isfinite(l.b) && isfinite(l.lo) && isfinite(l.hi);
  }
  // exclusive block scan of maxima
  __shared__ double wsum[32];
  unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double incl = loc;
  for (int d = 1; d < 32; d <<= 1) {
    double o = __shfl_up_sync(0xFFFFFFFFu, incl, d);
    if (lane >= (unsigned)d) incl = dmax(incl, o);
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    unsigned nw = blockDim.x >> 5;
    double v = lane < nw ? wsum[lane] : 0.0;
    for (int d = 1; d < 32; d <<= 1) {
      double o = __shfl_up_sync(0xFFFFFFFFu, v, d);
      if (lane >= (unsigned)d) v = dmax(v, o);
    }
    if (lane < nw) wsum[lane] = v;
  }
  __syncthreads();
  double excl = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
  if (lane == 0) excl = 0.0;
  if (wid > 0) excl = dmax(excl, wsum[wid - 1]);
  // sequential pass over my range with the exclusive prefix
  double hprev = excl;
  for (uint32_t i = i0; i < i0 + per && i < L; ++i) {
    Leaf l = lv[i];
    if (cn[i] == 0) {
      l.lo = hprev;
      l.hi = hprev;
    } else {
      l.lo = dmax(l.lo, hprev);
      l.hi = dmax(l.hi, l.lo);
    }
    hprev = l.hi;
    lv[i] = l;
  }
  int allfin = __syncthreads_and(fin ? 1 : 0);
  if (threadIdx.x == 0) {
    double range = __dsub_rn(md.xmax, md.xmin);
    bool ok = allfin && isfinite(md.xmin) && isfinite(md.xmax) && isfinite(range) && isfinite(md.ra) &&
              isfinite(md.rb);
    md.ok = ok ? 1u : 0u;
  }
}

// --------------------------------------------------- learned pivots

// v(u) = F(key(u)) * P: continuous refinement value of ord u.
__device__ __forceinline__ double refine_value(const DModel& m, const Leaf* lv, uint64_t u, double P, int dt) {
  return __dmul_rn(model_F(m, lv, ord_value(u, dt)), P);
}

// The same value when the root is known to route u to leaf l (every ord of
// an item whose two ends route to l does: the root is monotone), so the
// root's FP64 evaluation is skipped.  Same operations as model_F after the
// routing, hence the same result.
__device__ __forceinline__ double refine_value_leaf(const DModel& m, const Leaf& l, uint64_t u, double P, int dt) {
  double xc = dmax(ord_value(u, dt), m.xmin);
  xc = dmin(xc, m.xmax);
  double f = leaf_eval(l, xc);
  f = dmax(f, l.lo);
  f = dmin(f, l.hi);
  return __dmul_rn(f, P);
}

// Evaluator of v for one item: through the root, or straight in the one
// leaf all of the item's ords route to.
struct ItemEval {
  const DModel& m;
  const Leaf* lv;
  Leaf one_leaf;
  bool one;
  double P;
  int dt;
  __device__ __forceinline__ double operator()(uint64_t u) const {
    return one ? refine_value_leaf(m, one_leaf, u, P, dt) : refine_value(m, lv, u, P, dt);
  }
};

// Smallest u in [lo, hi] with v(u) >= t, given v(lo) < t <= v(hi).  v is
// monotone in u, so any bracketing search is exact.  Interpolation steps
// (with a bisection every fourth step) also test the neighbour of the
// estimate, so an estimate within one ord of the pivot closes the bracket.
__device__ uint64_t search_pivot(const ItemEval& v, uint64_t lo, uint64_t hi, double t, double vlo, double vhi) {
  uint64_t L = lo, H = hi;
  double vL = vlo, vH = vhi;
  for (int it = 0; it < 256 && H - L > 1; ++it) {
    uint64_t span = H - L;
    uint64_t mid;
    bool interp = (it & 3) != 3 && vH > vL;
    if (interp) {
      // the estimate only steers the search (every probe is evaluated
      // exactly), so the fraction is formed in FP32 and applied in fixed
      // point: o = span * frac with frac in [0, 1) as a 32-bit fraction
      const float frac = fminf(fmaxf((float)__dsub_rn(t, vL) / (float)__dsub_rn(vH, vL), 0.0f), 0.99999994f);
      const uint64_t f32 = (uint64_t)(frac * 4294967296.0f);
      uint64_t o = (span >> 32) * f32 + (((span & 0xFFFFFFFFull) * f32) >> 32);
      if (o < 1) o = 1;
      if (o > span - 1) o = span - 1;
      mid = L + o;
    } else {
      mid = L + (span >> 1);
    }
    double vm = v(mid);
    if (vm >= t) {
      H = mid;
      vH = vm;
      if (interp && mid - 1 > L) {
        double v2 = v(mid - 1);
        if (v2 >= t) {
          H = mid - 1;
          vH = v2;
        } else {
          L = mid - 1;
          vL = v2;
        }
      }
    } else {
      L = mid;
      vL = vm;
      if (interp && mid + 1 < H) {
        double v2 = v(mid + 1);
        if (v2 >= t) {
          H = mid + 1;
          vH = v2;
        } else {
          L = mid + 1;
          vL = v2;
        }
      }
    }
  }
  return H;
}

// The bucket a refinement value v maps to: clamp(floor(v) - Bg, 0, B-1)
// (the same arithmetic as refine_id after its multiplication by P).
__device__ __forceinline__ uint32_t bucket_of_value(double v, double Bg, uint32_t B) {
  double t = floor(v);
  t = __dsub_rn(t, Bg);
  return clamp_index(t, B - 1);
}

// Leaf the root routes ord u to (the model clamps the key to [xmin, xmax]).
__device__ __forceinline__ uint32_t leaf_of_ord(const DModel& m, uint64_t u, int dt) {
  double x = ord_value(u, dt);
  double xc = dmax(x, m.xmin);
  xc = dmin(xc, m.xmax);
  return root_leaf(m, xc);
}

// Smallest u in (lo, hi] routed to leaf >= l, given leaf_of(lo) < l <= leaf_of(hi):
// invert the linear root for a guess, gallop to bracket it, bisect.  Root
// evaluations are a third of a full model evaluation.
__device__ uint64_t root_boundary(const DModel& m, uint32_t l, int dt, uint64_t lo, uint64_t hi) {
  uint64_t L = lo, H = hi;  // leaf_of(L) < l <= leaf_of(H)
  if (m.ra > 0.0) {
    double xr = m.rx0 + ((double)l / (double)m.L - m.rb) / m.ra;
    double xl = ord_value(lo, dt), xh = ord_value(hi, dt);
    if (xr > xl && xr < xh) {
      uint64_t g;
      if (dt) g = xr >= 18446744073709549568.0 ? ~0ull : (uint64_t)xr;
      else g = ord_of((uint64_t)__double_as_longlong(xr), 0);
      if (g > L && g < H) {
        if (leaf_of_ord(m, g, dt) >= l) {
          H = g;
          for (uint64_t step = 1; step <= (1ull << 20); step <<= 1) {
            uint64_t c = H - L > step ? H - step : L;
            if (c == L) break;
            if (leaf_of_ord(m, c, dt) < l) {
              L = c;
              break;
            }
            H = c;
          }
        } else {
          L = g;
          for (uint64_t step = 1; step <= (1ull << 20); step <<= 1) {
            uint64_t c = H - L > step ? L + step : H;
            if (c == H) break;
            if (leaf_of_ord(m, c, dt) >= l) {
              H = c;
              break;
            }
            L = c;
          }
        }
      }
    }
  }
  for (int it = 0; it < 70 && H - L > 1; ++it) {
    uint64_t mid = L + ((H - L) >> 1);
    if (leaf_of_ord(m, mid, dt) >= l) H = mid;
    else L = mid;
  }
  return H;
}

// Per-item quantities every pivot of the item needs.
struct PivotPrep {
  double vlo, vhi, xlo, xhi, invP;
  uint32_t kmin, kmax, l0, l1;
};

__device__ __forceinline__ void pivot_prep(const DModel& m, const Leaf* lv, const Item& it, double P, double Bg,
                                           uint32_t B, int dt, PivotPrep& q) {
  q.vlo = refine_value(m, lv, it.ord_lo, P, dt);
  q.vhi = refine_value(m, lv, it.ord_hi, P, dt);
  q.kmin = bucket_of_value(q.vlo, Bg, B);
  q.kmax = bucket_of_value(q.vhi, Bg, B);
  q.xlo = ord_value(it.ord_lo, dt);
  q.xhi = ord_value(it.ord_hi, dt);
  q.l0 = root_leaf(m, dmin(dmax(q.xlo, m.xmin), m.xmax));
  q.l1 = root_leaf(m, dmin(dmax(q.xhi, m.xmin), m.xmax));
  q.invP = 1.0 / P;
}

// Bracket state of one pivot search: v(L) < t <= v(H), the pivot in (L, H].
// near = 2: probe the guess held in step; < 0: gallop down from H by step;
// 1: gallop up from L; 0: search.
struct PivotWork {
  uint64_t L, H, step;
  double vL, vH, t;
  uint32_t j;
  int8_t near;
  uint8_t it;
};

// The start of pivot j of an item: trivial slots, then the analytic guess
// inside the leaf whose F-range reaches the target (the leaf model is
// linear, so x* = x0 + (t/P - b)/a lands within a few ord of the pivot).
// Returns true when T[j] is written, else sets up the search in w: the
// item's bracket with the guess as its first probe (near = 2).
__device__ __forceinline__ bool pivot_start(uint32_t j, uint32_t B, const PivotPrep& q, const DModel& m,
                                            const Leaf* lv, double Bg, uint64_t lo, uint64_t hi, int dt, uint64_t* T,
                                            PivotWork& w) {
  if (j >= B) {
    T[j] = ~0ull;
    return true;
  }
  if (j == 0) {
    T[0] = lo;
    return true;
  }
  if (j <= q.kmin) {
    T[j] = lo;
    return true;
  }
  if (j > q.kmax) {
    T[j] = hi;
    return true;
  }
  const double t = __dadd_rn((double)j, Bg);
  const uint64_t L = lo, H = hi;
  int near = 0;
  // target F; it steers the leaf choice and the analytic guess only, the
  // pivot itself is confirmed by exact evaluations
  const double tF = __dmul_rn(t, q.invP);
  uint32_t l0 = q.l0, l1 = q.l1;
  while (l0 < l1) {  // first leaf whose clamp maximum reaches tF
    uint32_t mid = (l0 + l1) >> 1;
    if (lv[mid].hi < tF) l0 = mid + 1;
    else l1 = mid;
  }
  const Leaf lf = lv[l0];
  uint64_t guess = 0;
  if (!(tF > lf.lo) && l0 > q.l0) {
    // the target is at or below this leaf's floor: F jumps over it where
    // the root starts routing to leaf l0, so that boundary is the pivot
    const uint64_t u = root_boundary(m, l0, dt, lo, hi);
    if (u > L && u <= H) guess = u;
  } else if (lf.a > 0.0) {
    // 1/a from an FP32 reciprocal refined by two Newton-Raphson steps
    // (r <- r + r (1 - a r)): an FP64 division costs several times as much
    // on this part, and the guess only steers the search (exact
    // evaluations confirm the pivot)
    const float af = (float)lf.a;
    double xs;
    if (af > 1e-30f && af < 1e30f) {
      double r = (double)__frcp_rn(af);
      r = __fma_rn(r, __fma_rn(-lf.a, r, 1.0), r);
      r = __fma_rn(r, __fma_rn(-lf.a, r, 1.0), r);
      xs = __fma_rn(__dsub_rn(tF, lf.b), r, lf.x0);
    } else {
      xs = lf.x0 + (tF - lf.b) / lf.a;
    }
    if (xs >= q.xlo && xs <= q.xhi) {
      uint64_t u;
      if (dt) u = xs >= 18446744073709549568.0 ? ~0ull : (uint64_t)xs;
      else u = ord_of((uint64_t)__double_as_longlong(xs), 0);
      if (u > L && u < H) guess = u;
    }
  }
  if (guess) {  // the first probe evaluates the guess, then the search gallops from it
    near = 2;
  }
  w.L = L;
  w.H = H;
  w.step = guess ? guess : 1;
  w.vL = q.vlo;
  w.vH = q.vhi;
  w.t = t;
  w.j = j;
  w.near = (int8_t)near;
  w.it = 0;
  return false;
}

// One probe of a pivot search.  The guess lands a few ord from the pivot
// (the model's FP64 roundings make v flat over a few ord), so the search
// first gallops away from it (steps 1, 2, 4, ...) to a tight bracket, then
// bisects; wide brackets (no usable guess) take interpolation steps with a
// bisection every fourth step.  Any bracketing search finds the same pivot.
__device__ __forceinline__ void pivot_probe(const ItemEval& ev, PivotWork& w) {
  if (w.near == 2) {  // the analytic guess, then a gallop away from it
    const uint64_t c = w.step;
    const double v = ev(c);
    w.step = 1;
    if (v >= w.t) {
      w.H = c;
      w.vH = v;
      w.near = -1;
    } else {
      w.L = c;
      w.vL = v;
      w.near = 1;
    }
    return;
  }
  uint64_t c = 0;
  if (w.near < 0) {
    c = w.H - w.L > w.step ? w.H - w.step : w.L;
    if (c == w.L) w.near = 0;
  } else if (w.near > 0) {
    c = w.H - w.L > w.step ? w.L + w.step : w.H;
    if (c == w.H) w.near = 0;
  }
  if (w.near == 0) {
    const uint64_t span = w.H - w.L;
    if (span > 64 && (w.it & 3) != 3 && w.vH > w.vL) {
      const float frac =
          fminf(fmaxf((float)__dsub_rn(w.t, w.vL) / (float)__dsub_rn(w.vH, w.vL), 0.0f), 0.99999994f);
      const uint64_t f32 = (uint64_t)(frac * 4294967296.0f);
      uint64_t o = (span >> 32) * f32 + (((span & 0xFFFFFFFFull) * f32) >> 32);
      if (o < 1) o = 1;
      if (o > span - 1) o = span - 1;
      c = w.L + o;
    } else {
      c = w.L + (span >> 1);
    }
    ++w.it;
  }
  const double v = ev(c);
  if (v >= w.t) {
    w.H = c;
    w.vH = v;
    if (w.near < 0) w.step <<= 1;
    else w.near = 0;
  } else {
    w.L = c;
    w.vL = v;
    if (w.near > 0) w.step <<= 1;
    else w.near = 0;
  }
}

constexpr uint32_t kPivotTPB = 256;
constexpr int kPivotRounds = 96;

// One thread per pivot slot j of each listed item.  When a block lies inside
// one item (nb_pad a multiple of the block size) the item's end values are
// evaluated once per block, and the pivots whose guess did not confirm are
// pooled: each round every pooled search takes one probe and the unfinished
// ones are packed again, so the FP64 pipe (the bound here) runs full warps
// instead of warps in which a few lanes gallop.  Other blocks search per
// thread.
__device__ __forceinline__ void pivots_block(uint64_t blk, Plan* plans, const Item* items, const uint32_t* list,
                                             uint32_t nlist, uint32_t nb_pad, const DModel* models,
                                             const Leaf* leaves, uint64_t* __restrict__ pivots, const RunParams& rp) {
  __shared__ PivotPrep s_prep;
  __shared__ PivotWork s_w[2][kPivotTPB];
  __shared__ uint32_t s_n[2];
  const uint64_t g = blk * (uint64_t)blockDim.x + threadIdx.x;
  const bool pooled = nb_pad % blockDim.x == 0;
  if (pooled) {  // uniform: the whole block is in range and in one item
    if (g >= (uint64_t)nlist * nb_pad) return;
    if (threadIdx.x == 0) {
      const uint32_t pi0 = list[(uint32_t)(g / nb_pad)];
      const Plan& p0 = plans[pi0];
      const DModel m0 = models[p0.model];
      pivot_prep(m0, leaves + m0.leaf_off, items[pi0], p0.P, p0.Bg, rp.B, rp.dt, s_prep);
      s_n[0] = 0;
      s_n[1] = 0;
    }
    __syncthreads();
  } else if (g >= (uint64_t)nlist * nb_pad) {
    return;
  }
  const uint32_t li = (uint32_t)(g / nb_pad), j = (uint32_t)(g % nb_pad);
  const uint32_t pi = list[li];
  Plan& pl = plans[pi];
  const Item& it = items[pi];
  uint64_t* T = pivots + pl.tab_off;
  const uint32_t B = rp.B;
  const DModel m = models[pl.model];
  const Leaf* lv = leaves + m.leaf_off;
  const double P = pl.P, Bg = pl.Bg;
  PivotPrep q;
  if (pooled) q = s_prep;
  else pivot_prep(m, lv, it, P, Bg, B, rp.dt, q);
  if (j == 0) {
    pl.kmax = q.kmax;
    pl.nb = B;
    pl.nb_pad = nb_pad;
  }
  const ItemEval ev{m, lv, lv[q.l0], q.l0 == q.l1, P, rp.dt};
  PivotWork w;
  const bool done = pivot_start(j, B, q, m, lv, Bg, it.ord_lo, it.ord_hi, rp.dt, T, w);
  if (!pooled) {
    if (!done) {
      for (int r = 0; r < kPivotRounds && w.H - w.L > 1 && w.near != 0; ++r) pivot_probe(ev, w);
      T[j] = search_pivot(ev, w.L, w.H, w.t, w.vL, w.vH);
    }
    return;
  }
  if (!done) s_w[0][atomicAdd(&s_n[0], 1u)] = w;
  __syncthreads();
  int cur = 0;
  for (int r = 0; r < kPivotRounds; ++r) {
    const uint32_t n = s_n[cur];
    if (n == 0) break;  // uniform
    if (threadIdx.x < n) {
      PivotWork x = s_w[cur][threadIdx.x];
      pivot_probe(ev, x);
      if (x.H - x.L > 1) s_w[cur ^ 1][atomicAdd(&s_n[cur ^ 1], 1u)] = x;
      else T[x.j] = x.H;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_n[cur] = 0;  // the next round's destination
    cur ^= 1;
    __syncthreads();
  }
  // searches still open after the round limit finish on their own
  if (threadIdx.x < s_n[cur]) {
    const PivotWork& x = s_w[cur][threadIdx.x];
    T[x.j] = search_pivot(ev, x.L, x.H, x.t, x.vL, x.vH);
  }
}

// Blocks of nb_pad / blockDim.x pivot slots per listed item.  With bd (a
// device-planned batch) the list length is read on the device and the grid
// strides over the blocks.
__global__ void __launch_bounds__(kPivotTPB) k_learned_pivots(Plan* plans, const Item* items, const uint32_t* list,
                                                              uint32_t nlist, uint32_t nb_pad, const DModel* models,
                                                              const Leaf* leaves, uint64_t* __restrict__ pivots,
                                                              RunParams rp, const BatchDesc* bd) {
  pdl_wait();
  if (bd) nlist = bd->nrefine;
  const uint64_t nblk = ((uint64_t)nlist * nb_pad + blockDim.x - 1) / blockDim.x;
  for (uint64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    pivots_block(blk, plans, items, list, nlist, nb_pad, models, leaves, pivots, rp);
    __syncthreads();  // the block's shared search pool is reused by its next block of slots
  }
}

// Classify the candidates' own samples with their learned pivots (sample
// imbalance test).  Block (x, c) takes a stride of candidate c's samples:
// the candidate's pivot table and a histogram live in shared memory, and
// the block adds its histogram to the candidate's counts at the end.
__global__ void k_imbalance_count(FitArgs a, const uint64_t* __restrict__ pivots,
                                  unsigned long long* __restrict__ cnt, uint32_t nbp_max) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* sT = reinterpret_cast<uint64_t*>(smem);
  uint32_t* sH = reinterpret_cast<uint32_t*>(sT + nbp_max);
  const uint32_t c = blockIdx.y;
  const Plan& pl = a.plans[a.cand[c]];
  if (!a.models[pl.model].ok) return;  // uniform across the block
  const uint32_t nbp = pl.nb_pad;
  for (uint32_t j = threadIdx.x; j < nbp; j += blockDim.x) {
    sT[j] = pivots[pl.tab_off + j];
    sH[j] = 0;
  }
  __syncthreads();
  const uint64_t S = a.cand_soff[c + 1] - a.cand_soff[c];
  const uint64_t* samp = a.samp + pl.sample_off;
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < S; j += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t b = pivot_count(sT, nbp, samp[j]);
    b = b < pl.kmax ? b : pl.kmax;
    atomicAdd(&sH[b], 1u);
  }
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < nbp; j += blockDim.x)
    if (sH[j]) atomicAdd(&cnt[pl.cnt_off + j], (unsigned long long)sH[j]);
}

__global__ void k_imbalance_max(FitArgs a, unsigned long long* __restrict__ cnt) {
  pdl_wait();
  uint32_t c = blockIdx.x;
  Plan& pl = a.plans[a.cand[c]];
  unsigned long long mx = 0;
  for (uint32_t b = threadIdx.x; b < pl.nb_pad; b += blockDim.x) {
    unsigned long long v = cnt[pl.cnt_off + b];
    mx = v > mx ? v : mx;
    cnt[pl.cnt_off + b] = 0;
  }
  for (int d = 16; d > 0; d >>= 1) {
    unsigned long long o = __shfl_down_sync(0xFFFFFFFFu, mx, d);
    mx = o > mx ? o : mx;
  }
  __shared__ unsigned long long wm[32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long r = 0;
    for (unsigned w = 0; w < blockDim.x / 32; ++w) r = wm[w] > r ? wm[w] : r;
    if (a.models[pl.model].ok) pl.imb = r;
  }
}

// Alg. 5 BuildPartitionModel: RMI iff the input is large and the sample has
// few duplicates (and, in AUTO, the sample is not badly imbalanced).
__global__ void k_decide(FreshArgs f, const DModel* models, RunParams rp) {
  pdl_wait();
  uint32_t fi = blockIdx.x * blockDim.x + threadIdx.x;
  if (fi >= f.nfresh) return;
  uint32_t pi = f.fresh[fi];
  Plan& pl = f.plans[pi];
  const Item& it = f.items[pi];
  bool learned = false;
  bool want = false;
  if (it.kind != KIND_FORCE_SPLITTER && pl.want) {
    if (rp.partitioner == LS_PART_LEARNED) {
      want = true;
    } else if (rp.partitioner == LS_PART_AUTO) {
      double frac = __ddiv_rn(__ull2double_rn(pl.dups), __ull2double_rn((uint64_t)pl.S));
      want = (it.n >= rp.min_learned_n) && (frac <= rp.dup_frac);
    }
  }
  if (!want) pl.imb = 0;  // Alg. 5 never fits a model it does not want
  if (want && models[pl.model].ok) {
    {
      learned = true;
      if (rp.partitioner == LS_PART_AUTO) {
        double thr = __dmul_rn(rp.tau, __ull2double_rn((uint64_t)pl.S));
        thr = __ddiv_rn(thr, (double)rp.B);
        thr = dmax(thr, 16.0);
        if (__ull2double_rn(pl.imb) > thr) learned = false;
      }
    }
  }
  if (learned) {
    pl.decision = LS_DEC_LEARNED;
    pl.cls = (rp.classify_mode == LS_CLASSIFY_TREE)        ? CLS_TREE
             : (rp.classify_mode == LS_CLASSIFY_DIRECT)    ? CLS_DIRECT
             : (rp.classify_mode == LS_CLASSIFY_DIRECTORY) ? CLS_DIR
                                                           : CLS_GUESS;
  } else {
    pl.decision = LS_DEC_SPLITTER;  // refined to SPLITTER_EQ by the table build
    pl.model = -1;
  }
}

// SampleSort splitters from the sorted sample (Sec. 2.4): B_s - 1 equally
// spaced sample elements; equality buckets if two splitters coincide (or
// forced).  Written as exact pivots: bucket = #{j : T[j] <= ord}.
__global__ void __launch_bounds__(1024) k_splitter_build(FreshArgs f, const uint64_t* __restrict__ samp,
                                                         uint64_t* __restrict__ pivots, RunParams rp) {
  pdl_wait();
  uint32_t pi = f.fresh[blockIdx.x];
  Plan& pl = f.plans[pi];
  const Item& it = f.items[pi];
  if (pl.decision == LS_DEC_LEARNED) return;
  __shared__ uint64_t spl[LS_MAX_FANOUT];
  __shared__ uint16_t pos[LS_MAX_FANOUT];
  __shared__ uint32_t wtot[32];
  __shared__ int s_dup;
  uint64_t S = pl.S;
  const uint64_t* s = samp + pl.sample_off;
  bool force = it.kind == KIND_FORCE_SPLITTER;
  uint32_t bsmax = rp.bs_max;
  if (!force && rp.partitioner == LS_PART_AUTO && rp.bs_auto < bsmax) bsmax = rp.bs_auto;
  uint32_t bs = 1;
  while ((uint64_t)bs * 2 <= bsmax && (uint64_t)bs * 2 <= S && bs * 2 <= LS_MAX_FANOUT) bs *= 2;
  if (bs < 2) bs = 2;
  uint32_t ns = bs - 1;
  if (threadIdx.x == 0) s_dup = 0;
  __syncthreads();
  for (uint32_t k = threadIdx.x; k < ns; k += blockDim.x) spl[k] = s[((uint64_t)(k + 1) * S) / bs];
  __syncthreads();
  for (uint32_t k = threadIdx.x + 1; k < ns; k += blockDim.x)
    if (spl[k] == spl[k - 1]) s_dup = 1;
  __syncthreads();
  bool eq = s_dup || force;
  uint64_t* T = pivots + pl.tab_off;
  uint64_t lo = it.ord_lo, hi = it.ord_hi;
  uint32_t nb;
  uint32_t npiv;  // pivots T[1..npiv]
  if (eq) {
    // unique positions: exclusive scan of "new value" flags (4 per thread max)
    uint32_t per = (ns + blockDim.x - 1) / blockDim.x;
    uint32_t k0 = threadIdx.x * per;
    uint32_t cntl = 0;
    for (uint32_t k = k0; k < k0 + per && k < ns; ++k) cntl += (k == 0 || spl[k] != spl[k - 1]);
    unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = cntl;
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t o = __shfl_up_sync(0xFFFFFFFFu, incl, d);
      if (lane >= (unsigned)d) incl += o;
    }
    if (lane == 31) wtot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      unsigned nw = blockDim.x >> 5;
      uint32_t v = lane < nw ? wtot[lane] : 0;
      for (int d = 1; d < 32; d <<= 1) {
        uint32_t o = __shfl_up_sync(0xFFFFFFFFu, v, d);
        if (lane >= (unsigned)d) v += o;
      }
      if (lane < nw) wtot[lane] = v;
    }
    __syncthreads();
    uint32_t excl = incl - cntl + (wid > 0 ? wtot[wid - 1] : 0);
    for (uint32_t k = k0; k < k0 + per && k < ns; ++k) {
      if (k == 0 || spl[k] != spl[k - 1]) pos[excl++] = (uint16_t)k;
    }
    uint32_t m = wtot[(blockDim.x >> 5) - 1];
    __syncthreads();
    nb = 2 * m + 1;
    npiv = 2 * m;
    for (uint32_t q = threadIdx.x; q < m; q += blockDim.x) {
      uint64_t u = spl[pos[q]];
      T[2 * q + 1] = u;
      T[2 * q + 2] = (u == ~0ull) ? ~0ull : u + 1;  // u + 1 overflow: never reached
    }
  } else {
    nb = bs;
    npiv = ns;
    for (uint32_t k = threadIdx.x; k < ns; k += blockDim.x) {
      uint64_t u = spl[k];
      T[k + 1] = (u == ~0ull) ? ~0ull : u + 1;
    }
  }
  __syncthreads();
  // kmax = number of pivots a key <= hi can reach (pivots are sorted):
  // u_q counts iff u_q <= hi, u_q + 1 counts iff u_q < hi.
  uint32_t cnt_le = 0;
  if (eq) {
    uint32_t m = (nb - 1) / 2;
    for (uint32_t q = threadIdx.x; q < m; q += blockDim.x) {
      uint64_t u = spl[pos[q]];
      cnt_le += (u <= hi) + (u < hi);
    }
  } else {
    for (uint32_t k = threadIdx.x; k < ns; k += blockDim.x) cnt_le += (spl[k] < hi);
  }
  __shared__ uint32_t s_k;
  if (threadIdx.x == 0) s_k = 0;
  __syncthreads();
  for (int d = 16; d > 0; d >>= 1) cnt_le += __shfl_down_sync(0xFFFFFFFFu, cnt_le, d);
  if ((threadIdx.x & 31) == 0 && cnt_le) atomicAdd(&s_k, cnt_le);
  __syncthreads();
  uint32_t kmax = s_k;
  uint32_t nb_pad = 2;
  while (nb_pad < nb) nb_pad <<= 1;
  for (uint32_t j = threadIdx.x; j < nb_pad; j += blockDim.x) {
    if (j == 0) T[0] = lo;
    else if (j > npiv || j > kmax) T[j] = ~0ull;
    else if (T[j] < lo) T[j] = lo;
  }
  if (threadIdx.x == 0) {
    pl.nb = nb;
    pl.nb_pad = nb_pad;
    pl.kmax = kmax;
    pl.decision = eq ? LS_DEC_SPLITTER_EQ : LS_DEC_SPLITTER;
    pl.cls = (rp.classify_mode == LS_CLASSIFY_DIRECTORY) ? CLS_DIR : CLS_TREE;
    pl.model = -1;
  }
}

__global__ void k_dir_build(Plan* plans, uint32_t nplans, uint32_t cells, const uint64_t* __restrict__ pivots,
                            uint16_t* __restrict__ dirs) {
  pdl_wait();
  uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  uint64_t per = (uint64_t)cells + 1;
  if (g >= (uint64_t)nplans * per) return;
  uint32_t pi = (uint32_t)(g / per), c = (uint32_t)(g % per);
  Plan& pl = plans[pi];
  if (pl.cls != CLS_DIR) return;
  const uint64_t* T = pivots + pl.tab_off;
  uint32_t kmax = pl.kmax;
  uint64_t dlo, dhi;
  uint32_t shift = 0;
  if (kmax == 0) {
    dlo = ~0ull;
    dhi = ~0ull;
  } else {
    dlo = T[1];
    dhi = T[kmax];
    uint64_t span = dhi - dlo;
    uint32_t lc = 31 - __clz(cells);
    uint32_t bl = span ? 64 - __clzll((long long)span) : 0;
    shift = bl > lc ? bl - lc : 0;
  }
  uint16_t* D = dirs + pl.dir_off;
  uint32_t v;
  if (kmax == 0) {
    v = 0;
  } else {
    uint64_t add = shift >= 64 ? 0 : ((uint64_t)c << shift);
    uint64_t x = (add > ~0ull - dlo) ? ~0ull : dlo + add;
    v = pivot_count(T, pl.nb_pad, x);
    v = v < kmax ? v : kmax;
  }
  D[c] = (uint16_t)v;
  if (c == 0) {
    pl.dir_lo = dlo;
    pl.dir_hi = dhi;
    pl.dir_shift = shift;
    pl.dir_cells = cells;
  }
}

// ------------------------------------------------ fit forward / backward

struct GradScratch {
  double* rl;      // leaf residuals
  double* Xl;      // leaf X
  double* rr;      // root residuals
  double* Xr;      // root X
  uint64_t* key;   // (leaf << 32) | j
  uint64_t* key2;  // sort scratch
  uint64_t* segoff;   // 2
  uint64_t* cpre;     // 2
  uint32_t* lstart;   // L + 1
  uint64_t* lch;      // L + 1 chunk counts / prefix
  uint64_t* lchp;     // L + 1
  uint64_t* stmp;     // scan tmp
  size_t stmp_elems;
  double* part;       // 2 * (S/256 + L + 2) * 2
  double* rpart;      // 4 * (S/256 + 1)
};

__global__ void k_grad_fwd(const DModel* mp, const Leaf* leaves, const uint64_t* __restrict__ bits, uint64_t S,
                           int dt, double* pred, double* resid, GradScratch g) {
  pdl_wait();
  uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (j >= S) return;
  DModel m = *mp;
  double x = key_value(bits[j], dt);
  double xc = dmax(x, m.xmin);
  xc = dmin(xc, m.xmax);
  uint32_t i = root_leaf(m, xc);
  Leaf l = leaves[i];
  double y = __ddiv_rn(__ull2double_rn(j), __ull2double_rn(S));
  double X = __dsub_rn(xc, l.x0);
  double p = __dmul_rn(l.a, X);
  p = __dadd_rn(p, l.b);
  double r = __dsub_rn(p, y);
  if (pred) pred[j] = p;
  if (resid) resid[j] = r;
  g.rl[j] = r;
  g.Xl[j] = X;
  double XR = __dsub_rn(xc, m.rx0);
  double pr = __dmul_rn(m.ra, XR);
  pr = __dadd_rn(pr, m.rb);
  g.rr[j] = __dsub_rn(pr, y);
  g.Xr[j] = XR;
  g.key[j] = ((uint64_t)i << 32) | j;
}

__global__ void k_grad_leaf_starts(const uint64_t* __restrict__ sorted, uint64_t S, uint32_t L, uint32_t* lstart) {
  pdl_wait();
  uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (q >= S) return;
  uint32_t lf = (uint32_t)(sorted[q] >> 32);
  lf = lf < L ? lf : L - 1;
  if (q == 0) {
    for (uint32_t i = 0; i <= lf; ++i) lstart[i] = 0;
  } else {
    uint32_t prev = (uint32_t)(sorted[q - 1] >> 32);
    prev = prev < L ? prev : L - 1;
    for (uint32_t i = prev + 1; i <= lf; ++i) lstart[i] = (uint32_t)q;
  }
  if (q == S - 1)
    for (uint32_t i = lf + 1; i <= L; ++i) lstart[i] = (uint32_t)S;
}

__global__ void k_grad_chunk_count(const uint32_t* lstart, uint32_t L, uint64_t* lch) {
  pdl_wait();
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > L) return;
  lch[i] = (i == L) ? 0 : ((uint64_t)(lstart[i + 1] - lstart[i]) + kChunk - 1) / kChunk;
}

__global__ void k_grad_leaf_partials(const uint64_t* __restrict__ sorted, const uint32_t* lstart, const uint64_t* lchp,
                                     uint32_t L, uint64_t bound, GradScratch g) {
  pdl_wait();
  uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (q >= lchp[L] || q >= bound) return;
  uint32_t i = find_seg(lchp, L, q);
  uint64_t k = q - lchp[i];
  uint64_t st = lstart[i], en = lstart[i + 1];
  uint64_t a0 = st + k * kChunk;
  uint64_t a1 = a0 + kChunk < en ? a0 + kChunk : en;
  double prx = 0.0, pr = 0.0;
  for (uint64_t t = a0; t < a1; ++t) {
    uint64_t j = sorted[t] & 0xFFFFFFFFull;
    double rx = __dmul_rn(g.rl[j], g.Xl[j]);
    prx = __dadd_rn(prx, rx);
    pr = __dadd_rn(pr, g.rl[j]);
  }
  g.part[q] = prx;
  g.part[bound + q] = pr;
}

__global__ void k_grad_leaf_finish(const uint64_t* lchp, uint32_t L, uint64_t bound, uint64_t S, GradScratch g,
                                   double* grad_a, double* grad_b) {
  pdl_wait();
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  uint64_t p0 = lchp[i], m = lchp[i + 1] - p0;
  double srx = thread_tree_sum(g.part + p0, m);
  double sr = thread_tree_sum(g.part + bound + p0, m);
  double Sd = __ull2double_rn(S);
  if (grad_a) grad_a[i] = __ddiv_rn(__dmul_rn(2.0, srx), Sd);
  if (grad_b) grad_b[i] = __ddiv_rn(__dmul_rn(2.0, sr), Sd);
}

__global__ void k_grad_root_partials(uint64_t S, uint64_t nch, GradScratch g) {
  pdl_wait();
  uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (c >= nch) return;
  uint64_t a0 = c * kChunk, a1 = a0 + kChunk < S ? a0 + kChunk : S;
  double prx = 0.0, pr = 0.0;
  for (uint64_t j = a0; j < a1; ++j) {
    double rx = __dmul_rn(g.rr[j], g.Xr[j]);
    prx = __dadd_rn(prx, rx);
    pr = __dadd_rn(pr, g.rr[j]);
  }
  g.rpart[c] = prx;
  g.rpart[nch + c] = pr;
}

__global__ void k_grad_root_finish(uint64_t S, uint64_t nch, GradScratch g, double* grad_root) {
  pdl_wait();
  double srx = block_tree_sum(g.rpart, g.rpart + 2 * nch, nch);
  double sr = block_tree_sum(g.rpart + nch, g.rpart + 3 * nch, nch);
  if (threadIdx.x == 0 && grad_root) {
    double Sd = __ull2double_rn(S);
    grad_root[0] = __ddiv_rn(__dmul_rn(2.0, srx), Sd);
    grad_root[1] = __ddiv_rn(__dmul_rn(2.0, sr), Sd);
  }
}

// FP32 image of model slot `slot`: thread per leaf, one extra for the root.
__device__ __forceinline__ void fmodel_one(const DModel* models, const Leaf* leaves, int32_t slot, uint32_t i,
                                           uint32_t L, FModel* fm, FLeaf* fl, FClamp* fc) {
  const DModel& m = models[slot];
  if (i < L) {
    Leaf l = leaves[m.leaf_off + i];
    fl[m.leaf_off + i] = make_float4(__double2float_rn(l.x0), __double2float_rn(l.a), __double2float_rn(l.b), 0.0f);
    if (fc) fc[m.leaf_off + i] = make_float2(__double2float_rn(l.lo), __double2float_rn(l.hi));
  } else if (i == L) {
    FModel f;
    f.xminf = __double2float_rn(m.xmin);
    f.xmaxf = __double2float_rn(m.xmax);
    f.rx0f = __double2float_rn(m.rx0);
    f.raL = __double2float_rn(__dmul_rn(m.ra, (double)m.L));
    f.rbL = __double2float_rn(__dmul_rn(m.rb, (double)m.L));
    f.L = m.L;
    f.leaf_off = m.leaf_off;
    fm[slot] = f;
  }
}

__global__ void k_fmodel(const DModel* models, const Leaf* leaves, const int32_t* slots, uint32_t nslots,
                         uint32_t L, FModel* fm, FLeaf* fl, FClamp* fc) {
  pdl_wait();
  uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (g >= (uint64_t)nslots * (L + 1)) return;
  uint32_t c = (uint32_t)(g / (L + 1)), i = (uint32_t)(g % (L + 1));
  fmodel_one(models, leaves, slots[c], i, L, fm, fl, fc);
}

__global__ void k_fmodel_fit(FitArgs a) {
  pdl_wait();
  uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (g >= (uint64_t)a.ncand * (a.L + 1)) return;
  uint32_t c = (uint32_t)(g / (a.L + 1)), i = (uint32_t)(g % (a.L + 1));
  fmodel_one(a.models, a.leaves, a.plans[a.cand[c]].model, i, a.L, a.fmodels, a.fleaves, a.fclamps);
}

}  // namespace

// ===================================================== host launchers

uint64_t* segmented_sort_u64(uint64_t* a, uint64_t* b, const uint64_t* d_off, const uint64_t* d_chunk_prefix,
                             uint32_t nseg, uint64_t total_chunks, uint64_t max_len, cudaStream_t st,
                             uint64_t* launches) {
  if (total_chunks == 0) return a;
  pdl_launch(k_sort_chunks, (unsigned)total_chunks, kSortTPB, 0, st, a, d_off, d_chunk_prefix, nseg);
  ++*launches;
  uint64_t* cur = a;
  uint64_t* oth = b;
  for (uint64_t w = kSortChunk; w < max_len; w *= 2) {
    pdl_launch(k_merge_pass, (unsigned)total_chunks, kMergeTPB, 0, st, cur, oth, d_off, d_chunk_prefix, nseg, w);
    ++*launches;
    uint64_t* t = cur;
    cur = oth;
    oth = t;
  }
  return cur;
}

void launch_sample_gather(const FreshArgs& f, const RunParams& rp, uint64_t* samp, cudaStream_t st) {
  if (!f.total_samples) return;
  pdl_launch(k_sample_gather, grid_for(f.total_samples), kTPB, 0, st, f, rp, samp);
}

void launch_sample_keys(const uint64_t* keys, uint64_t n, uint64_t S, uint64_t h, uint64_t* out, cudaStream_t st) {
  if (!S) return;
  pdl_launch(k_sample_keys, grid_for(S), kTPB, 0, st, keys, n, S, h, out);
}

void launch_dups(const FreshArgs& f, const uint64_t* samp, cudaStream_t st) {
  if (!f.total_samples) return;
  pdl_launch(k_dups, grid_for(f.total_samples), kTPB, 0, st, f, samp);
}

void launch_fit(const FitArgs& a, const RunParams& rp, cudaStream_t st, uint64_t* launches) {
  if (!a.ncand) return;
  pdl_launch(k_fit_root_partials, grid_for(a.total_rchunks * 32, 128), 128, 0, st, a, rp);
  {
    static size_t set[64] = {};
    const size_t sm = (size_t)4 * kRootSmemChunks * sizeof(double);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && set[dev] < sm) {
      cudaFuncSetAttribute(k_fit_root_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      set[dev] = sm;
    }
    pdl_launch(k_fit_root_finish, a.ncand, 1024, sm, st, a, rp);
  }
  cudaMemsetAsync(a.leaf_start, 0, (size_t)a.ncand * (a.L + 1) * sizeof(uint32_t), st);
  pdl_launch(k_fit_route_leaf, grid_for(a.total_cand_samples), kTPB, 0, st, a, rp, a.leaf_of);
  pdl_launch(k_fit_route_starts, grid_for(a.total_cand_samples), kTPB, 0, st, a, a.leaf_of);
  uint64_t tot = (uint64_t)a.ncand * a.L;
  pdl_launch(k_fit_leaf_chunk_count, grid_for(tot + 1), kTPB, 0, st, a);
  launch_scan_exclusive_u64(a.lchunk_cnt, a.lchunk_prefix, tot, a.scan_tmp, a.scan_tmp_elems, st);
  pdl_launch(k_fit_leaf_partials, grid_for(a.lchunk_bound * 32, 128), 128, 0, st, a, rp);
  pdl_launch(k_fit_leaf_finish, grid_for(tot * 32, 128), 128, 0, st, a, rp, a.leaf_cnt);
  pdl_launch(k_fit_leaf_lane, grid_for(tot, 128), 128, 0, st, a, rp, a.leaf_cnt);
  pdl_launch(k_fit_monotone, a.ncand, 1024, 0, st, a, a.leaf_cnt);
  pdl_launch(k_fmodel_fit, grid_for((uint64_t)a.ncand * (a.L + 1)), kTPB, 0, st, a);
  *launches += 14;
}

void launch_fmodel(const DModel* models, const Leaf* leaves, const int32_t* slots, uint32_t nslots, uint32_t L,
                   FModel* fm, FLeaf* fl, cudaStream_t st, FClamp* fc) {
  if (!nslots) return;
  pdl_launch(k_fmodel, grid_for((uint64_t)nslots * (L + 1)), kTPB, 0, st, models, leaves, slots, nslots, L, fm, fl, fc);
}

void launch_learned_pivots(Plan* plans, const Item* items, const uint32_t* list, uint32_t nlist, uint32_t nb_pad,
                           const DModel* models, const Leaf* leaves, uint64_t* pivots, const RunParams& rp,
                           cudaStream_t st, const BatchDesc* bd) {
  // with bd, nlist bounds the list length read on the device
  if (!nlist) return;
  uint64_t n = (uint64_t)nlist * nb_pad;
  uint32_t tpb = nb_pad >= kPivotTPB ? kPivotTPB : 128;  // pooled blocks when tpb divides nb_pad
  if (!bd) {
    // short lists (a root, the few items of a deep level): smaller blocks
    // spread the searches over more SMs' FP64 pipes (the rounds of a block
    // are a chain of FP64 evaluations)
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    while (tpb > 32 && n / tpb < 2ull * (uint64_t)(sms > 0 ? sms : 1) && nb_pad % (tpb / 2) == 0) tpb /= 2;
  }
  // one block per block of slots of the largest list (blocks past the
  // device-side list end return at once): the search rounds of a block are
  // synchronised, so blocks are scheduled as slots free up rather than
  // strided over
  pdl_launch(k_learned_pivots, grid_for(n, tpb), tpb, 0, st, plans, items, list, nlist, nb_pad, models, leaves, pivots,
             rp, bd);
}

void launch_imbalance(const FitArgs& a, uint64_t* pivots, unsigned long long* cnt_pool, const RunParams& rp,
                      cudaStream_t st, uint64_t* launches) {
  (void)rp;
  if (!a.ncand) return;
  // candidates' tables are at most nb_pad_max entries (the learned fanout, padded)
  const uint32_t nbp_max = a.nbp_max;
  const size_t sm = (size_t)nbp_max * 12;
  static size_t set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (sm > set[dev]) {
    cudaFuncSetAttribute(k_imbalance_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    set[dev] = sm;
  }
  const uint64_t per = (a.total_cand_samples + a.ncand - 1) / a.ncand;  // mean samples per candidate
  uint64_t gx = (per + kTPB * 8 - 1) / (kTPB * 8);
  gx = gx < 1 ? 1 : (gx > 256 ? 256 : gx);
  pdl_launch(k_imbalance_count, dim3((unsigned)gx, a.ncand), kTPB, sm, st, a, pivots, cnt_pool, nbp_max);
  pdl_launch(k_imbalance_max, a.ncand, kTPB, 0, st, a, cnt_pool);
  *launches += 2;
}

void launch_decide(const FreshArgs& f, const DModel* models, const RunParams& rp, cudaStream_t st) {
  if (!f.nfresh) return;
  pdl_launch(k_decide, grid_for(f.nfresh, 128), 128, 0, st, f, models, rp);
}

void launch_splitter_build(const FreshArgs& f, const uint64_t* samp, uint64_t* pivots, const RunParams& rp,
                           cudaStream_t st) {
  if (!f.nfresh) return;
  pdl_launch(k_splitter_build, f.nfresh, 1024, 0, st, f, samp, pivots, rp);
}

void launch_dir_build(Plan* plans, uint32_t nplans, uint32_t cells, const uint64_t* pivots, uint16_t* dirs,
                      cudaStream_t st) {
  if (!nplans) return;
  uint64_t n = (uint64_t)nplans * (cells + 1);
  pdl_launch(k_dir_build, grid_for(n), kTPB, 0, st, plans, nplans, cells, pivots, dirs);
}

size_t fit_grad_scratch_bytes(uint64_t S, uint32_t L) {
  uint64_t nch = (S + kChunk - 1) / kChunk;
  uint64_t bound = nch + L + 2;
  size_t b = 0;
  b += 4 * S * sizeof(double);          // rl Xl rr Xr
  b += 2 * S * sizeof(uint64_t);        // key key2
  b += 4 * sizeof(uint64_t);            // segoff cpre
  b += (L + 1) * sizeof(uint32_t) + 64;
  b += 2 * (L + 1) * sizeof(uint64_t);
  b += scan_tmp_elems(L + 1) * sizeof(uint64_t);
  b += 2 * bound * sizeof(double);
  b += 4 * (nch + 1) * sizeof(double);
  return b + 1024;
}

void launch_fit_grad(const DModel* model, const Leaf* leaves, const uint64_t* sample_bits, uint64_t S, int dt,
                     double* pred, double* resid, double* grad_a, double* grad_b, double* grad_root, void* scratch,
                     size_t scratch_bytes, cudaStream_t st) {
  (void)scratch_bytes;
  if (S == 0) return;
  DModel hm;
  cudaMemcpyAsync(&hm, model, sizeof(DModel), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  uint32_t L = hm.L;
  uint64_t nch = (S + kChunk - 1) / kChunk;
  uint64_t bound = nch + L + 2;
  char* p = static_cast<char*>(scratch);
  auto take = [&](size_t bytes) {
    char* r = p;
    p += (bytes + 255) & ~size_t(255);
    return r;
  };
  GradScratch g;
  g.rl = reinterpret_cast<double*>(take(S * 8));
  g.Xl = reinterpret_cast<double*>(take(S * 8));
  g.rr = reinterpret_cast<double*>(take(S * 8));
  g.Xr = reinterpret_cast<double*>(take(S * 8));
  g.key = reinterpret_cast<uint64_t*>(take(S * 8));
  g.key2 = reinterpret_cast<uint64_t*>(take(S * 8));
  g.segoff = reinterpret_cast<uint64_t*>(take(16));
  g.cpre = reinterpret_cast<uint64_t*>(take(16));
  g.lstart = reinterpret_cast<uint32_t*>(take((L + 1) * 4));
  g.lch = reinterpret_cast<uint64_t*>(take((L + 1) * 8));
  g.lchp = reinterpret_cast<uint64_t*>(take((L + 1) * 8));
  g.stmp_elems = scan_tmp_elems(L + 1);
  g.stmp = reinterpret_cast<uint64_t*>(take(g.stmp_elems * 8));
  g.part = reinterpret_cast<double*>(take(2 * bound * 8));
  g.rpart = reinterpret_cast<double*>(take(4 * (nch + 1) * 8));
  const Leaf* lv = leaves + hm.leaf_off;
  pdl_launch(k_grad_fwd, grid_for(S), kTPB, 0, st, model, lv, sample_bits, S, dt, pred, resid, g);
  uint64_t hoff[2] = {0, S};
  uint64_t hcp[2] = {0, (S + kSortChunk - 1) / kSortChunk};
  cudaMemcpyAsync(g.segoff, hoff, sizeof hoff, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(g.cpre, hcp, sizeof hcp, cudaMemcpyHostToDevice, st);
  uint64_t dummy = 0;
  uint64_t* sorted = segmented_sort_u64(g.key, g.key2, g.segoff, g.cpre, 1, hcp[1], S, st, &dummy);
  pdl_launch(k_grad_leaf_starts, grid_for(S), kTPB, 0, st, sorted, S, L, g.lstart);
  pdl_launch(k_grad_chunk_count, grid_for(L + 1), kTPB, 0, st, g.lstart, L, g.lch);
  launch_scan_exclusive_u64(g.lch, g.lchp, L, g.stmp, g.stmp_elems, st);
  pdl_launch(k_grad_leaf_partials, grid_for(bound), kTPB, 0, st, sorted, g.lstart, g.lchp, L, bound, g);
  pdl_launch(k_grad_leaf_finish, grid_for(L), kTPB, 0, st, g.lchp, L, bound, S, g, grad_a, grad_b);
  pdl_launch(k_grad_root_partials, grid_for(nch), kTPB, 0, st, S, nch, g);
  pdl_launch(k_grad_root_finish, 1, 1024, 0, st, S, nch, g, grad_root);
  cudaStreamSynchronize(st);  // hoff / hcp live on this stack frame
}

}  // namespace lsg
