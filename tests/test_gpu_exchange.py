"""The one-exchange sample sort with the library's own backend on the GPU:
ls_sample, ls_fit, ls_classify and ls_sort through the C ABI on each rank,
the exchange through gloo on the host.  One rank, and two ranks sharing the
GPU (each runs its own kernels; nothing waits on the other rank's kernels).
The result must be the sorted union of the shards, bit for bit."""
import os
import tempfile

import numpy as np
import pytest

import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def np_ord(x):
    if x.dtype == np.uint64:
        return x.copy()
    b = x.view(np.uint64)
    return np.where((b >> np.uint64(63)).astype(bool), ~b, b | np.uint64(1 << 63))


def _shard(name, rank):
    return datagen.generate(name, [1_500_000, 2_600_000][rank % 2], 60 + rank)


def _worker(rank, world, port, name, outdir):
    import torch.distributed as dist

    import paper_2307_08637_gb300 as lsg
    from paper_2307_08637_gb300 import exchange
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    ctx = lsg.Context(0)
    x = torch.from_numpy(_shard(name, rank)).to("cuda:0")
    out, info = exchange.exchange_sort(x, exchange.LibraryBackend(ctx), seed=11)
    np.save(os.path.join(outdir, f"out{rank}.npy"), out.cpu().numpy())
    np.save(os.path.join(outdir, f"bounds{rank}.npy"), np.array(info.bounds + [info.sample_size]))
    ctx.close()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,name", [(1, "normal"), (2, "normal"), (2, "skewed_u64")])
def test_exchange_sort_library_backend(world, name):
    import torch.multiprocessing as mp
    port = 29850 + 10 * world + (3 if name == "normal" else 7)
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_worker, args=(world, port, name, d), nprocs=world, join=True)
        outs = [np.load(os.path.join(d, f"out{r}.npy")) for r in range(world)]
        bds = [np.load(os.path.join(d, f"bounds{r}.npy")) for r in range(world)]
    allx = np.concatenate([_shard(name, r) for r in range(world)])
    ref = allx[np.argsort(np_ord(allx), kind="stable")]
    assert np.array_equal(np.concatenate(outs).view(np.uint64), ref.view(np.uint64))
    assert all(np.array_equal(bds[0], b) for b in bds)  # one replicated model and range split
    if world == 2:
        assert abs(outs[0].size - allx.size / 2) < 0.05 * allx.size
