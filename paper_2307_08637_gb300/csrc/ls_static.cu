// ls_static.cu -- ls_classify_static: bucket classification that allocates no
// device memory.
//
// Some callers cannot call cudaMalloc at the point where they need to
// classify keys: an application whose memory pool already owns the device's
// memory (a database buffer manager, a framework's caching allocator), or a
// latency-critical path where cudaMalloc's possible device-wide
// synchronisation is not acceptable.  This entry point keeps all of its
// scratch (device copy of the model, exact pivots, directory, plan) in one
// file-scope device array of fixed size instead of context memory.
//
// The array is shared by every call in the process and keeps the last call's
// contents; each call overwrites everything it reads before reading it.
// Calls that overlap on the GPU (different streams, or host threads racing)
// race on the array: serialise them.  The array occupies kStaticScratchBytes
// on every GPU that loads the library, until the process exits.
#include <cstddef>
#include <cstring>
#include <mutex>

#include "ls_kernels.h"

using namespace lsg;

namespace {

// Enough for every mode at every fanout up to LS_MAX_FANOUT (the largest
// layout, GUESS at 4096 leaves, needs about 274 KB).
constexpr size_t kStaticScratchBytes = 288 * 1024;
constexpr uint32_t kStaticDirBits = 13;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_classify_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

inline size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of g_classify_scratch on the current device (resolved once
// per device; the host-side symbol is only a stand-in, never a device address).
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_classify_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// Scratch layout for fanout B (all offsets 256-aligned).
struct StaticLayout {
  size_t model, leaves, item, plan, pivots, dir, list, fmodel, fleaves, slot, total;
};

StaticLayout static_layout(uint32_t B, uint32_t nb_pad, uint32_t cells) {
  StaticLayout l;
  size_t off = 0;
  l.model = off;
  off = up256(off + sizeof(DModel));
  l.leaves = off;
  off = up256(off + (size_t)B * sizeof(Leaf));
  l.item = off;
  off = up256(off + sizeof(Item));
  l.plan = off;
  off = up256(off + sizeof(Plan));
  l.pivots = off;
  off = up256(off + (size_t)nb_pad * 8);
  l.dir = off;
  off = up256(off + (size_t)(cells + 1) * 2);
  l.list = off;
  off = up256(off + 4);
  l.fmodel = off;
  off = up256(off + sizeof(FModel));
  l.fleaves = off;
  off = up256(off + (size_t)B * sizeof(FLeaf));
  l.slot = off;
  off = up256(off + 4);
  l.total = off;
  return l;
}

}  // namespace

extern "C" ls_status ls_classify_static(const ls_model* model, const void* d_keys, uint64_t n, ls_dtype dtype,
                                        uint32_t k, uint64_t g, int32_t mode, uint32_t* d_ids, uint64_t* d_hist,
                                        ls_stream_t stream) {
  if (!model || (!d_keys && n) || (dtype != LS_F64 && dtype != LS_U64)) return LS_EINVAL;
  if (model->L < 2 || model->L > LS_MAX_FANOUT || mode < LS_CLASSIFY_AUTO || mode > LS_CLASSIFY_GUESS)
    return LS_EINVAL;
  // B >= 2, so B^(k+1) > 2^50 for every k >= 50: reject those before the
  // power loop (k + 1 would also wrap at k = UINT32_MAX).
  if (k >= 50) return LS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t B = model->L;
  double P = 1.0;
  for (uint32_t i = 0; i <= k && P <= kRefineLimit; ++i) P = P * (double)B;
  if (P > kRefineLimit) return LS_EINVAL;
  const double Bg = (double)((uint64_t)B * g);
  uint32_t nbp = 1;
  while (nbp < B) nbp <<= 1;
  const uint32_t cells = 1u << kStaticDirBits;
  const StaticLayout lay = static_layout(B, nbp, cells);
  if (lay.total > kStaticScratchBytes) {
    set_error_detail("ls_classify_static: fanout %u needs %zu bytes of scratch, the static array holds %zu", B,
                     lay.total, kStaticScratchBytes);
    return LS_ENOMEM;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LS_ECUDA;
  void* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) return LS_ECUDA;
  char* b = static_cast<char*>(base);
  DModel* d_m = reinterpret_cast<DModel*>(b + lay.model);
  Leaf* d_l = reinterpret_cast<Leaf*>(b + lay.leaves);
  Item* d_it = reinterpret_cast<Item*>(b + lay.item);
  Plan* d_pl = reinterpret_cast<Plan*>(b + lay.plan);
  uint64_t* d_piv = reinterpret_cast<uint64_t*>(b + lay.pivots);
  uint16_t* d_dir = reinterpret_cast<uint16_t*>(b + lay.dir);
  uint32_t* d_list = reinterpret_cast<uint32_t*>(b + lay.list);
  FModel* d_fm = reinterpret_cast<FModel*>(b + lay.fmodel);
  FLeaf* d_fl = reinterpret_cast<FLeaf*>(b + lay.fleaves);
  int32_t* d_slot = reinterpret_cast<int32_t*>(b + lay.slot);

  // Host images of everything the kernels read; every field is written on
  // every call, so nothing from an earlier call is ever used.
  DModel dm;
  memset(&dm, 0, sizeof dm);
  dm.xmin = model->xmin;
  dm.xmax = model->xmax;
  dm.rx0 = model->root_x0;
  dm.ra = model->root_a;
  dm.rb = model->root_b;
  dm.L = B;
  dm.S = model->S;
  dm.leaf_off = 0;
  dm.ok = 1;
  if (cudaMemcpyAsync(d_m, &dm, sizeof dm, cudaMemcpyHostToDevice, st) != cudaSuccess) return LS_ECUDA;
  // the model's per-leaf arrays go straight into the leaf records (strided
  // copies: no host-side staging buffer either)
  const double* src[5] = {model->leaf_x0, model->leaf_a, model->leaf_b, model->leaf_lo, model->leaf_hi};
  const size_t fld[5] = {offsetof(Leaf, x0), offsetof(Leaf, a), offsetof(Leaf, b), offsetof(Leaf, lo),
                         offsetof(Leaf, hi)};
  for (int q = 0; q < 5; ++q) {
    if (cudaMemcpy2DAsync(reinterpret_cast<char*>(d_l) + fld[q], sizeof(Leaf), src[q], sizeof(double), sizeof(double),
                          B, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return LS_ECUDA;
  }
  if (d_hist && cudaMemsetAsync(d_hist, 0, B * sizeof(uint64_t), st) != cudaSuccess) return LS_ECUDA;
  if (mode == LS_CLASSIFY_DIRECT) {
    launch_direct_classify(d_m, d_l, static_cast<const uint64_t*>(d_keys), n, dtype, P, Bg, B, d_ids,
                           reinterpret_cast<unsigned long long*>(d_hist), st);
  } else {
    Item it;
    memset(&it, 0, sizeof it);
    if (dtype == LS_U64) {
      it.ord_lo = 0;
      it.ord_hi = ~0ull;
    } else {
      it.ord_lo = kOrdMinF64;
      it.ord_hi = kOrdMaxF64;
    }
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
    if (cudaMemcpyAsync(d_it, &it, sizeof it, cudaMemcpyHostToDevice, st) != cudaSuccess) return LS_ECUDA;
    if (cudaMemcpyAsync(d_pl, &pl, sizeof pl, cudaMemcpyHostToDevice, st) != cudaSuccess) return LS_ECUDA;
    if (cudaMemcpyAsync(d_list, &zero, 4, cudaMemcpyHostToDevice, st) != cudaSuccess) return LS_ECUDA;
    if (cudaMemcpyAsync(d_slot, &zero, 4, cudaMemcpyHostToDevice, st) != cudaSuccess) return LS_ECUDA;
    RunParams rp;
    memset(&rp, 0, sizeof rp);
    rp.B = B;
    rp.dt = dtype;
    launch_learned_pivots(d_pl, d_it, d_list, 1, nbp, d_m, d_l, d_piv, rp, st);
    launch_dir_build(d_pl, 1, cells, d_piv, d_dir, st);
    if (mode == LS_CLASSIFY_GUESS) launch_fmodel(d_m, d_l, d_slot, 1, B, d_fm, d_fl, st);
    launch_table_classify(d_pl, d_piv, d_dir, static_cast<const uint64_t*>(d_keys), n, dtype, d_ids,
                          reinterpret_cast<unsigned long long*>(d_hist), nbp, cells, st, d_fm, d_fl);
  }
  if (cudaGetLastError() != cudaSuccess) return LS_ECUDA;
  // the host images above live on this stack frame: finish the copies
  if (cudaStreamSynchronize(st) != cudaSuccess) return LS_ECUDA;
  return LS_OK;
}
