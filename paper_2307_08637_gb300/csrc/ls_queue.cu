// ls_queue.cu -- the device work queue of the level loop.
//
// Below the root level, a sort under REFINE_GLOBAL only ever refines the
// root's model or takes the radix split (no bucket draws a sample, Sec. 2.2),
// so every later level can be planned on the device: the items of a level
// are (segment, bucket) pairs in a device array, K2 appends the next level's
// items to another, and one planner block turns up to kBatchItems of them
// into the plans, chunk map, chunk runs, scatter runs and pivot list of a
// batch.  The kernels of the batch read their counts from the planner's
// descriptor, so the batch needs no host round trip; the loop-control kernel
// decides on the device whether another batch follows (the condition of a
// CUDA graph's while node, or a flag the host reads).  Items that would draw
// a sample (below a splitter tree) are handed back to the host planner.
#include "ls_kernels.h"

namespace lsg {

namespace {

constexpr int kPlanTPB = 1024;
static_assert(kBatchItems == 2 * kPlanTPB, "the planner holds two items per thread");
constexpr int kPlanWarps = kPlanTPB / 32;

// Block-wide exclusive scan (thread order) of K values per thread; every
// thread gets the totals.  One barrier: each warp scans the warp totals
// itself.  sh holds kPlanWarps * K words and is not reused by the caller.
template <int K>
__device__ __forceinline__ void plan_scan(uint32_t (&v)[K], uint32_t (&tot)[K], uint32_t* sh) {
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) inc[k] = v[k];
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, inc[k], d);
      if (lane >= (unsigned)d) inc[k] += o;
    }
  }
  if (lane == 31)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[wid * K + k] = inc[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    uint32_t x = sh[lane * K + k];  // warp `lane`'s total (kPlanWarps == 32)
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, x, d);
      if (lane >= (unsigned)d) x += o;
    }
    const uint32_t before = __shfl_sync(0xFFFFFFFFu, x, (wid + 31) & 31);
    tot[k] = __shfl_sync(0xFFFFFFFFu, x, 31);
    v[k] = inc[k] - v[k] + (wid > 0 ? before : 0u);
  }
}
static_assert(kPlanWarps == 32, "plan_scan scans one warp total per lane");

__device__ __forceinline__ uint32_t pow2ceil_dev(uint32_t x) { return x <= 1 ? 1u : 1u << (32 - __clz(x - 1)); }

// B^e in FP64, stopping once past the refinement limit (the host's
// pow_exact, operation for operation).
__device__ __forceinline__ double pow_refine(uint32_t B, uint32_t e) {
  double P = 1.0;
  for (uint32_t i = 0; i < e && P <= kRefineLimit; ++i) P = __dmul_rn(P, (double)B);
  return P;
}

// One batch of the current level: switch levels when the current one is
// exhausted, take up to kBatchItems items, hand back those that draw a
// sample, and lay out the batch for its kernels.  One block.
__global__ void __launch_bounds__(kPlanTPB) k_plan_batch(PlanArgs a, RunParams rp, LoopHandles hs) {
  pdl_wait();
  __shared__ uint32_t sh1[kPlanWarps], sh7[kPlanWarps * 7];
  __shared__ unsigned long long s_sum[kPlanWarps];
  QueueState* q = a.q;
  uint64_t cur_n = q->cur_n, head = q->head;
  // the previous batch's spans have been sorted (the spans of the levels
  // planned on the host before the first batch are sorted with it)
  if (q->iter > 0 && threadIdx.x == 0) {
    a.ctr->n_base_small = 0;
    a.ctr->n_base_mid = 0;
    a.ctr->n_base_large = 0;
    a.ctr->n_copy = 0;
    a.ctr->n_fallback = 0;
  }
  if (head >= cur_n) {  // uniform: the level is done, the next one becomes current
    uint64_t nn = a.ctr->n_next;
    if (nn > a.icap) nn = a.icap;  // K2 has flagged the overflow; the loop stops after this batch
    const uint4* src = reinterpret_cast<const uint4*>(a.next);
    uint4* dst = reinterpret_cast<uint4*>(a.level);
    for (uint64_t w = threadIdx.x; w < nn * (sizeof(Item) / 16); w += blockDim.x) dst[w] = src[w];
    __syncthreads();  // every thread has read the counters before they are reset
    if (threadIdx.x == 0) {
      q->cur_n = nn;
      q->head = 0;
      a.ctr->n_next = 0;
    }
    cur_n = nn;
    head = 0;
  }
  const uint32_t k = (uint32_t)(cur_n - head < kBatchItems ? cur_n - head : kBatchItems);
  const uint32_t B = rp.B;
  // 1. keep the items planned here (refine and radix items), hand back the
  // rest; the kept ones keep their order
  Item its[2];
  bool kp[2] = {false, false};
  uint32_t keep[1] = {0}, nk1[1];
  unsigned long long nsum = 0;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const uint32_t idx = 2 * threadIdx.x + j;
    if (idx >= k) continue;
    its[j] = a.level[head + idx];
    const Item& it = its[j];
    kp[j] = it.kind == KIND_RADIX || (it.kind == KIND_REFINE && !beyond_refine_limit(B, (uint32_t)it.mk + 1u));
    if (kp[j]) {
      keep[0] += 1;
      nsum += it.n;
    } else {
      const unsigned long long slot = atomicAdd(&q->host_n, 1ull);
      if (slot < a.icap) a.hostq[slot] = it;
      else atomicExch(&a.ctr->overflow, 1ull);
    }
  }
  for (int d = 16; d > 0; d >>= 1) nsum += __shfl_xor_sync(0xFFFFFFFFu, nsum, d);
  if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = nsum;
  plan_scan<1>(keep, nk1, sh1);  // its barrier also publishes s_sum
  unsigned long long bkeys = 0;
  for (int w = 0; w < kPlanWarps; ++w) bkeys += s_sum[w];
  const uint32_t nk = nk1[0];
  // chunk size: 64Ki keys, halved (down to one tile) while the batch would
  // have fewer than kChunkSlots chunks (as the host planner does)
  uint64_t ck = kChunkKeys;
  while (ck > kTileKeys && bkeys / ck < kChunkSlots) ck >>= 1;
  // buffered-scatter runs: about an equal share of the run slots, at least a tile
  const uint64_t share = (bkeys + a.slots - 1) / a.slots;
  const uint64_t target = share > kTileKeys ? share : (uint64_t)kTileKeys;
  // 2. per kept item: chunks, chunk runs, multi-run flag, pivot search,
  // scatter runs; and the classifiers the batch uses
  uint32_t v[7] = {0, 0, 0, 0, 0, 0, 0}, tot[7];
  uint32_t nc[2] = {0, 0}, nr[2] = {0, 0};
  bool refine[2] = {false, false};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    if (!kp[j]) continue;
    const uint64_t n = its[j].n;
    nc[j] = (uint32_t)((n + ck - 1) / ck);
    nr[j] = (uint32_t)((n + target - 1) / target);
    refine[j] = its[j].kind == KIND_REFINE && rp.classify_mode != LS_CLASSIFY_DIRECT && n >= 4ull * B;
    v[0] += nc[j];
    v[1] += (nc[j] + kSegChunks - 1) / kSegChunks;
    v[2] += nc[j] > kSegChunks;
    v[3] += refine[j];
    v[4] += nr[j];
    v[5] += its[j].kind == KIND_REFINE && !refine[j];
    v[6] += its[j].kind == KIND_RADIX;
  }
  plan_scan<7>(v, tot, sh7);
  const bool fits = tot[0] <= a.chunk_cap && tot[1] <= a.seg_cap && tot[4] <= a.run_cap;
  if (!fits) {  // cannot happen with the workspace's capacities; stop the loop with an error
    if (threadIdx.x == 0) {
      atomicCAS(a.status, 0u, (unsigned)LS_ENOMEM);
      a.bd->nitems = 0;
      a.bd->nchunks = 0;
      a.bd->nsegs = a.bd->nmulti = a.bd->nruns = a.bd->nrefine = 0;
      q->head = head + k;
      if (hs.in_graph) {
        cudaGraphSetConditional(hs.pivots, 0);
        cudaGraphSetConditional(hs.k1, 0);
        if (hs.has_direct) cudaGraphSetConditional(hs.direct, 0);
        cudaGraphSetConditional(hs.radix, 0);
        cudaGraphSetConditional(hs.multi, 0);
      }
    }
    return;
  }
  // 3. items, plans, chunk map, chunk runs, scatter runs, pivot list
  uint32_t i = keep[0];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    if (!kp[j]) continue;
    const Item& it = its[j];
    a.bitems[i] = it;
    Plan pl;
    memset(&pl, 0, sizeof pl);
    pl.chunk_begin = v[0];
    pl.cnt_off = (uint64_t)i * a.nbc;
    pl.tab_off = (uint64_t)i * a.nbc;
    pl.dir_off = (uint64_t)i * (a.cells + 1);
    pl.model = -1;
    if (it.kind == KIND_RADIX) {
      const uint32_t nb = radix_buckets(it.mk);
      pl.decision = LS_DEC_RADIX;
      pl.cls = CLS_RADIX;
      pl.nb = nb;
      pl.nb_pad = nb;
      pl.kmax = nb - 1;
      pl.dir_shift = radix_shift(it.mk);
    } else {
      pl.P = pow_refine(B, (uint32_t)it.mk + 1u);
      pl.Bg = (double)((uint64_t)B * it.mg);
      pl.model = it.model;
      pl.decision = LS_DEC_LEARNED;
      pl.nb = B;
      pl.nb_pad = pow2ceil_dev(B);
      pl.kmax = B - 1;
      pl.cls = !refine[j]                                   ? CLS_DIRECT
               : rp.classify_mode == LS_CLASSIFY_TREE       ? CLS_TREE
               : rp.classify_mode == LS_CLASSIFY_DIRECTORY  ? CLS_DIR
                                                             : CLS_GUESS;
    }
    a.plans[i] = pl;
    for (uint32_t c = 0; c < nc[j]; ++c) a.chunk_plan[v[0] + c] = i;
    const uint32_t nsg = (nc[j] + kSegChunks - 1) / kSegChunks;
    for (uint32_t g = 0; g < nsg; ++g) {
      ChunkSeg sg;
      sg.c0 = v[0] + (uint64_t)g * kSegChunks;
      sg.nch = nc[j] - g * kSegChunks < kSegChunks ? nc[j] - g * kSegChunks : kSegChunks;
      sg.plan = i;
      sg.first = v[1];
      sg.pad = 0;
      a.segs[v[1] + g] = sg;
    }
    if (nc[j] > kSegChunks) a.multi[v[2]] = make_uint2(v[1], nsg);
    if (refine[j]) a.reflist[v[3]] = i;
    for (uint32_t r = 0; r < nr[j]; ++r) {
      BufRun br;
      br.off = it.n * r / nr[j];
      br.len = it.n * (r + 1) / nr[j] - br.off;
      br.plan = i;
      br.pad = 0;
      br.pad1 = 0;
      a.runs[v[4] + r] = br;
    }
    v[0] += nc[j];
    v[1] += nsg;
    v[2] += nc[j] > kSegChunks;
    v[3] += refine[j];
    v[4] += nr[j];
    ++i;
  }
  if (threadIdx.x == 0) {
    BatchDesc d;
    memset(&d, 0, sizeof d);
    d.nchunks = tot[0];
    d.chunk_keys = ck;
    d.keys = bkeys;
    d.nitems = nk;
    d.nsegs = tot[1];
    d.nmulti = tot[2];
    d.nrefine = tot[3];
    d.nruns = tot[4];
    *a.bd = d;
    a.chunk_ctr[0] = 0;
    a.chunk_ctr[1] = 0;
    q->head = head + k;
    if (hs.in_graph) {  // inside the graph: skip the kernels this batch does not need
      cudaGraphSetConditional(hs.pivots, tot[3] > 0);
      cudaGraphSetConditional(hs.k1, tot[3] > 0);
      if (hs.has_direct) cudaGraphSetConditional(hs.direct, tot[5] > 0);
      cudaGraphSetConditional(hs.radix, tot[6] > 0);
      cudaGraphSetConditional(hs.multi, tot[2] > 0);
    }
  }
}

// Counts of the batch's items, zeroed before K1 adds to them.
__global__ void k_zero_counts(const BatchDesc* bd, const Plan* plans, unsigned long long* counts) {
  pdl_wait();
  const uint32_t ni = bd->nitems;
  for (uint32_t i = blockIdx.x; i < ni; i += gridDim.x) {
    const Plan& pl = plans[i];
    for (uint32_t b = threadIdx.x; b < pl.nb_pad; b += blockDim.x) counts[pl.cnt_off + b] = 0;
  }
}

// End of a batch, after its scatter: continue while items remain, no list
// overflowed, the device status is clean and the iteration limit is not
// reached; inside the graph, also say which span lists the batch filled.
__global__ void k_batch_end(QueueState* q, const LevelCounters* ctr, const unsigned int* status, LoopHandles hs,
                            unsigned long long max_iter) {
  pdl_wait();
  const bool err = ctr->overflow != 0 || *status != 0;
  const unsigned long long it = q->iter + 1;
  q->iter = it;
  unsigned int c = (!err && (q->head < q->cur_n || ctr->n_next > 0)) ? 1u : 0u;
  if (c && it >= max_iter) {
    c = 0;
    q->err = 1;
  }
  q->cont = c;
  if (hs.in_graph) {
    cudaGraphSetConditional(hs.small, ctr->n_base_small > 0 || ctr->n_base_mid > 0);
    cudaGraphSetConditional(hs.large, ctr->n_base_large > 0);
    cudaGraphSetConditional(hs.copy, ctr->n_copy > 0);
    cudaGraphSetConditional(hs.fallback, ctr->n_fallback > 0);
    cudaGraphSetConditional(hs.loop, c);
  }
}

}  // namespace

void launch_plan_batch(const PlanArgs& a, const RunParams& rp, const LoopHandles& h, cudaStream_t st) {
  pdl_launch(k_plan_batch, 1, kPlanTPB, 0, st, a, rp, h);
}

void launch_zero_counts(const BatchDesc* bd, const Plan* plans, unsigned long long* counts, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  pdl_launch(k_zero_counts, (unsigned)(sms > 0 ? sms : 1) * 4, 256, 0, st, bd, plans, counts);
}

void launch_batch_end(QueueState* q, const LevelCounters* ctr, const unsigned int* status, const LoopHandles& h,
                      unsigned long long max_iter, cudaStream_t st) {
  pdl_launch(k_batch_end, 1, 1, 0, st, q, ctr, status, h, max_iter);
}

}  // namespace lsg
