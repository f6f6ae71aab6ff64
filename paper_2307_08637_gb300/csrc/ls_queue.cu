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
// thread gets the totals.  sh holds kPlanWarps * K words.
template <int K>
__device__ void plan_scan(uint32_t (&v)[K], uint32_t (&tot)[K], uint32_t* sh) {
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
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      uint32_t x = sh[lane * K + k];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= (unsigned)d) x += o;
      }
      sh[lane * K + k] = x;  // inclusive over warps
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const uint32_t before = wid > 0 ? sh[(wid - 1) * K + k] : 0u;
    tot[k] = sh[(kPlanWarps - 1) * K + k];
    v[k] = inc[k] - v[k] + before;
  }
  __syncthreads();  // sh is reused by the next scan
}

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
__global__ void __launch_bounds__(kPlanTPB) k_plan_batch(PlanArgs a, RunParams rp) {
  pdl_wait();
  __shared__ uint32_t sh[kPlanWarps * 5];
  __shared__ unsigned long long s_sum[kPlanWarps];
  QueueState* q = a.q;
  uint64_t cur_n = q->cur_n, head = q->head;
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
  // 1. keep the items planned here (refine and radix items), hand back the rest
  Item mine[2];
  bool kp[2] = {false, false};
  uint32_t keep[1] = {0}, nk1[1];
  unsigned long long nsum = 0;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const uint32_t idx = 2 * threadIdx.x + j;
    if (idx >= k) continue;
    mine[j] = a.level[head + idx];
    const Item& it = mine[j];
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
  plan_scan<1>(keep, nk1, sh);
  {
    uint32_t o = keep[0];
#pragma unroll
    for (int j = 0; j < 2; ++j)
      if (kp[j]) a.bitems[o++] = mine[j];
  }
  for (int d = 16; d > 0; d >>= 1) nsum += __shfl_xor_sync(0xFFFFFFFFu, nsum, d);
  if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = nsum;
  __syncthreads();  // kept items and warp sums are visible to the block
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
  // 2. per kept item: chunks, chunk runs, multi-run flag, pivot search, scatter runs
  uint32_t v[5] = {0, 0, 0, 0, 0}, tot[5];
  Item its[2];
  uint32_t nc[2] = {0, 0}, nr[2] = {0, 0};
  bool refine[2] = {false, false};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const uint32_t i = 2 * threadIdx.x + j;
    if (i >= nk) continue;
    its[j] = a.bitems[i];
    const uint64_t n = its[j].n;
    nc[j] = (uint32_t)((n + ck - 1) / ck);
    nr[j] = (uint32_t)((n + target - 1) / target);
    refine[j] = its[j].kind == KIND_REFINE && rp.classify_mode != LS_CLASSIFY_DIRECT && n >= 4ull * B;
    v[0] += nc[j];
    v[1] += (nc[j] + kSegChunks - 1) / kSegChunks;
    v[2] += nc[j] > kSegChunks;
    v[3] += refine[j];
    v[4] += nr[j];
  }
  plan_scan<5>(v, tot, sh);
  const bool fits = tot[0] <= a.chunk_cap && tot[1] <= a.seg_cap && tot[4] <= a.run_cap;
  if (!fits) {  // cannot happen with the workspace's capacities; stop the loop with an error
    if (threadIdx.x == 0) {
      atomicCAS(a.status, 0u, (unsigned)LS_ENOMEM);
      a.bd->nitems = 0;
      a.bd->nchunks = 0;
      a.bd->nsegs = a.bd->nmulti = a.bd->nruns = a.bd->nrefine = 0;
      q->head = head + k;
    }
    return;
  }
  // 3. plans, chunk map, chunk runs, scatter runs, pivot list
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const uint32_t i = 2 * threadIdx.x + j;
    if (i >= nk) continue;
    const Item& it = its[j];
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

// End of a batch: its finished spans have been sorted, so the span lists
// start again; continue while items remain, no list overflowed, the device
// status is clean and the iteration limit is not reached.
__global__ void k_loop_ctl(QueueState* q, LevelCounters* ctr, const unsigned int* status,
                           cudaGraphConditionalHandle h, unsigned long long max_iter) {
  pdl_wait();
  ctr->n_base_small = 0;
  ctr->n_base_large = 0;
  ctr->n_copy = 0;
  ctr->n_fallback = 0;
  const bool err = ctr->overflow != 0 || *status != 0;
  const unsigned long long it = q->iter + 1;
  q->iter = it;
  unsigned int c = (!err && (q->head < q->cur_n || ctr->n_next > 0)) ? 1u : 0u;
  if (c && it >= max_iter) {
    c = 0;
    q->err = 1;
  }
  q->cont = c;
  if (h) cudaGraphSetConditional(h, c);
}

}  // namespace

void launch_plan_batch(const PlanArgs& a, const RunParams& rp, cudaStream_t st) {
  pdl_launch(k_plan_batch, 1, kPlanTPB, 0, st, a, rp);
}

void launch_zero_counts(const BatchDesc* bd, const Plan* plans, unsigned long long* counts, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  pdl_launch(k_zero_counts, (unsigned)(sms > 0 ? sms : 1) * 4, 256, 0, st, bd, plans, counts);
}

void launch_loop_ctl(QueueState* q, LevelCounters* ctr, const unsigned int* status, cudaGraphConditionalHandle h,
                     unsigned long long max_iter, cudaStream_t st) {
  pdl_launch(k_loop_ctl, 1, 1, 0, st, q, ctr, status, h, max_iter);
}

}  // namespace lsg
