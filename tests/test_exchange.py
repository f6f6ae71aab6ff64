"""The one-exchange sample sort across ranks (paper_2307_08637_gb300.exchange)
on two gloo ranks on the CPU.  The ranks run the exchange logic with a
backend built from the CPU oracle (the model fit and bucket function, pinned
elsewhere) and numpy's sort; the check is the plain definition: the ranks'
outputs, concatenated in rank order, are the sorted union of the shards, and
every rank holds about N / P keys."""
import os
import tempfile

import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")

from paper_2307_08637_gb300 import exchange  # noqa: E402

B = 1000


def np_ord(x):
    if x.dtype == np.uint64:
        return x.copy()
    b = x.view(np.uint64)
    return np.where((b >> np.uint64(63)).astype(bool), ~b, b | np.uint64(1 << 63))


class OracleBackend:
    """CPU backend: the oracle's sample positions, fit and bucket function."""

    def sample(self, keys, S, seed):
        x = keys.numpy()
        pos = oracle.sample_positions(seed, x.size, S).astype(np.int64) if S < x.size else np.arange(x.size)
        return torch.from_numpy(x[pos].copy())

    def fit(self, sample):
        x = sample.numpy()
        m, ok = oracle.fit(x[np.argsort(np_ord(x), kind="stable")], B)
        assert ok
        return m

    def histogram(self, model, keys):
        _, h = oracle.classify(model, keys.numpy(), B)
        return torch.from_numpy(h.astype(np.int64))

    def sort(self, keys):
        x = keys.numpy()
        return torch.from_numpy(x[np.argsort(np_ord(x), kind="stable")].copy())


def _shard(dist_name, rank):
    n = [150_000, 260_000, 90_000][rank % 3]
    return datagen.generate(dist_name, n, 40 + rank)


def _worker(rank, world, port, dist_name, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x = torch.from_numpy(_shard(dist_name, rank))
    out, info = exchange.exchange_sort(x, OracleBackend(), seed=7)
    np.save(os.path.join(outdir, f"out{rank}.npy"), out.numpy())
    np.save(os.path.join(outdir, f"info{rank}.npy"), np.array([info.received, info.sample_size] + info.bounds))
    dist.destroy_process_group()


@pytest.mark.parametrize("dist_name", ["normal", "lognormal", "skewed_u64"])
def test_two_rank_exchange_sort(dist_name):
    import torch.multiprocessing as mp
    world = 2
    port = 29600 + hash(dist_name) % 200
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_worker, args=(world, port, dist_name, d), nprocs=world, join=True)
        outs = [np.load(os.path.join(d, f"out{r}.npy")) for r in range(world)]
        infos = [np.load(os.path.join(d, f"info{r}.npy")) for r in range(world)]
    allx = np.concatenate([_shard(dist_name, r) for r in range(world)])
    got = np.concatenate(outs)
    ref = allx[np.argsort(np_ord(allx), kind="stable")]
    assert np.array_equal(got.view(np.uint64), ref.view(np.uint64))
    # every rank fitted on the same gathered sample and agreed on the ranges
    assert all(np.array_equal(infos[0][1:], i[1:]) for i in infos)
    assert infos[0][1] == sum(max(256, int(np.ceil(0.01 * _shard(dist_name, r).size))) for r in range(world))
    # balance: each rank within one bucket of N / P
    N = allx.size
    _, h = oracle.classify(OracleBackend().fit(torch.from_numpy(np.concatenate(
        [OracleBackend().sample(torch.from_numpy(_shard(dist_name, r)), max(256, int(np.ceil(0.01 * _shard(dist_name, r).size))),
                                exchange.rank_seed(7, r)).numpy() for r in range(world)]))), allx, B)
    for r in range(world):
        assert abs(int(infos[r][0]) - N / world) <= int(h.max()) + 1


def test_bucket_bounds_balance_and_cover():
    rng = np.random.default_rng(3)
    for world in (1, 2, 3, 8):
        c = rng.integers(0, 50, 1000)
        bd = exchange.bucket_bounds(list(c), world)
        assert bd[0] == 0 and bd[-1] == 1000 and all(a <= b for a, b in zip(bd, bd[1:]))
        tot = int(c.sum())
        for j in range(world):
            share = int(c[bd[j]:bd[j + 1]].sum())
            assert abs(share - tot / world) <= 2 * int(c.max())
    assert exchange.bucket_bounds([0, 0, 0], 2) == [0, 0, 3]
