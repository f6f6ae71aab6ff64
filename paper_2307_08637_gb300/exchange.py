"""One-exchange sample sort of a key array spread over ranks.

The paper's parallel results come down to balance: buckets of equal size are
what let the parallel sort scale (Sec. 5), and a learned CDF model gives
balanced buckets from a small sample (Sec. 3, Table 1).  Across GPUs the
same idea sorts an array that is spread over the ranks with one exchange:

1. every rank draws a sample of its shard (``Sample`` of Alg. 2-5, the
   library's ``ls_sample``);
2. the samples are gathered on every rank and every rank fits the same RMI
   on the same bytes (``ls_fit`` on the gathered sample, which it sorts
   itself), so the model is replicated without sending it;
3. each rank classifies its shard (``ls_classify``, histogram only) and the
   B-bucket histograms are summed over the ranks;
4. rank j receives the contiguous bucket range whose global count prefix
   crosses j N / P, so every rank gets about N / P keys;
5. each rank sorts its shard (``ls_sort``), which makes the keys bound for
   each rank contiguous, sends them with one all-to-all, and sorts what it
   received.

The concatenation of the ranks' outputs in rank order is the sorted array.
The data path is the library's kernels plus the collectives; the collective
tensors live on the CUDA device under NCCL and on the host under gloo.

Every step that touches keys goes through a backend object, so the exchange
logic can also run on ranks without a GPU (the tests give it one):
``sample(keys, S, seed)``, ``fit(sample) -> model``, ``histogram(model, keys)
-> int64 counts[B]``, ``sort(keys) -> keys``.  ``LibraryBackend`` is the
backend of the product: the C ABI through the ctypes binding.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

GOLDEN = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def rank_seed(seed: int, rank: int) -> int:
    """Sampling stream of one rank: the ranks' streams differ by whole
    multiples of 2^40 draws, so they never overlap for shards below 2^40 keys."""
    return (seed + rank * (GOLDEN << 40)) & M64


def bucket_bounds(counts, world: int) -> list[int]:
    """Rank j takes buckets [bounds[j], bounds[j+1]): bounds[j] is the first
    bucket whose exclusive count prefix reaches j * N / world (integer
    arithmetic), so ranks get contiguous, balanced bucket ranges."""
    B = len(counts)
    total = int(sum(int(c) for c in counts))
    bounds = [0] * (world + 1)
    bounds[world] = B
    pre = 0
    b = 0
    for j in range(1, world):
        goal = (j * total + world - 1) // world  # ceil(j N / P)
        while b < B and pre < goal:
            pre += int(counts[b])
            b += 1
        bounds[j] = b
    return bounds


@dataclass
class ExchangeInfo:
    sample_size: int
    counts: list        # global B-bucket histogram
    bounds: list        # bucket range of each rank
    sent: list          # keys this rank sent to each rank
    received: int       # keys this rank holds after the exchange


class LibraryBackend:
    """The library's kernels on one CUDA device (C ABI via ctypes)."""

    def __init__(self, ctx, params=None):
        from . import ls
        self.ls = ls
        self.ctx = ctx
        self.p = params or ls.ls_params_default()

    def sample(self, keys, S: int, seed: int):
        return self.ls.ls_sample(self.ctx, keys, S, seed)

    def fit(self, sample):
        p = self.ls.ls_params_default(fanout=self.p.fanout, sample_rate=1.0,
                                      partitioner=self.ls.LS_PART_LEARNED, seed=self.p.seed)
        m, _, _ = self.ls.ls_fit(self.ctx, sample.contiguous(), p)
        return m

    def histogram(self, model, keys):
        _, hist = self.ls.ls_classify(self.ctx, model, keys, want_ids=False)
        return hist

    def sort(self, keys):
        keys = keys.contiguous()
        if keys.numel() > 1:
            self.ls.ls_sort(self.ctx, keys, self.p)
        return keys


def _all_gather_var(t, group, dev):
    """all_gather of 1-D tensors of different lengths (padded to the longest)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n = torch.tensor([t.numel()], dtype=torch.int64, device=dev)
    ns = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(ns, n, group=group)
    ns = [int(x.item()) for x in ns]
    m = max(ns) if ns else 0
    buf = torch.zeros(m, dtype=torch.int64, device=dev)
    buf[:t.numel()] = t.view(torch.int64).to(dev)
    outs = [torch.zeros(m, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(outs, buf, group=group)
    return torch.cat([o[:k] for o, k in zip(outs, ns)])


def exchange_sort(keys, backend, *, sample_rate: float = 0.01, min_sample: int = 256, seed: int = 1,
                  group=None):
    """Sort the array whose shard on this rank is `keys` (1-D float64 or
    uint64 tensor); returns (this rank's part of the sorted array, info).
    Collective: every rank of `group` calls it."""
    import torch
    import torch.distributed as dist

    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    coll = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" \
        else torch.device("cpu")
    n = keys.numel()
    S = min(n, max(int(math.ceil(sample_rate * n)), min_sample)) if n else 0
    s = backend.sample(keys, S, rank_seed(seed, rank))
    gathered = _all_gather_var(s, group, coll)
    sample = gathered.to(keys.device).view(keys.dtype)
    model = backend.fit(sample)
    counts = backend.histogram(model, keys).to(torch.int64)
    total = counts.to(coll).clone()
    dist.all_reduce(total, group=group)
    total_l = [int(x) for x in total.cpu().tolist()]
    bounds = bucket_bounds(total_l, world)
    local = [int(x) for x in counts.cpu().tolist()]
    send = [sum(local[bounds[j]:bounds[j + 1]]) for j in range(world)]
    srt = backend.sort(keys)
    scounts = torch.tensor(send, dtype=torch.int64, device=coll)
    rcounts = torch.empty(world, dtype=torch.int64, device=coll)
    dist.all_to_all_single(rcounts, scounts, group=group)
    recv_sizes = [int(x) for x in rcounts.cpu().tolist()]
    out = torch.empty(sum(recv_sizes), dtype=torch.int64, device=coll)
    dist.all_to_all_single(out, srt.view(torch.int64).to(coll), recv_sizes, send, group=group)
    mine = backend.sort(out.to(keys.device).view(keys.dtype))
    return mine, ExchangeInfo(sample_size=int(sample.numel()), counts=total_l, bounds=bounds, sent=send,
                              received=int(mine.numel()))
