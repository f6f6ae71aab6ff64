"""Key-value sort (ls_sort_pairs / ls_argsort): the keys come out exactly as
ls_sort and the oracle give them (same partition decisions), and the values
are the input values permuted by the stable argsort of the keys' ord image
(the plain definition: equal keys keep their input order)."""
import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2307_08637_gb300 as lsg  # noqa: E402


def ord_u64(x):
    b = x.view(np.uint64)
    if x.dtype == np.float64:
        return np.where(b >> np.uint64(63), ~b, b | np.uint64(1 << 63))
    return b


def stable_perm(x):
    return np.argsort(ord_u64(x), kind="stable")


@pytest.fixture(scope="module")
def ctx():
    c = lsg.Context(0)
    yield c
    c.close()


CASES = [("normal", 700_001, {}), ("lognormal", 300_000, {"basecase_threshold": 4096}),
         ("zipf", 500_000, {}), ("root_dups", 400_000, {"basecase_threshold": 4096}),
         ("two_dups", 300_000, {"partitioner": oracle.PART_SPLITTER}), ("skewed_u64", 600_000, {}),
         ("uniform01", 2**20, {"fanout": 1000, "basecase_threshold": 16}),
         ("mix_gauss", 250_000, {"recurse_model": oracle.RECURSE_RETRAIN}),
         ("normal", 200_000, {"max_depth": 1})]


@pytest.mark.parametrize("vbytes", [4, 8])
@pytest.mark.parametrize("dist,n,kw", CASES)
def test_pairs_match_stable_argsort_and_oracle(ctx, dist, n, kw, vbytes):
    x = datagen.generate(dist, n, 9)
    rng = np.random.default_rng(5)
    vals = rng.integers(0, 2**31 if vbytes == 4 else 2**62, size=n).astype(np.int32 if vbytes == 4 else np.int64)
    k = torch.from_numpy(x).to("cuda:0")
    v = torch.from_numpy(vals).to("cuda:0")
    st = lsg.ls_sort_pairs(ctx, k, v, lsg.ls_params_default(**kw))
    perm = stable_perm(x)
    assert np.array_equal(k.cpu().numpy().view(np.uint64), x[perm].view(np.uint64))
    assert np.array_equal(v.cpu().numpy(), vals[perm])
    out, rc, tr, _, _ = oracle.sort(x, oracle.params(**kw))
    assert rc == 0 and st.levels() == tr.levels() and st.root_decision == tr.root_decision


def test_argsort_edge_sizes(ctx):
    for n in (0, 1, 2, 3, 31, 33, 257, 4096, 4097, 65537):
        x = datagen.generate("root_dups", max(n, 1), n)[:n]
        k = torch.from_numpy(x.copy()).to("cuda:0")
        idx = lsg.ls_argsort(ctx, k)
        assert np.array_equal(idx.cpu().numpy(), stable_perm(x)), n


def test_argsort_all_equal_and_special_values(ctx):
    x = np.full(150_000, 2.5)
    k = torch.from_numpy(x.copy()).to("cuda:0")
    assert np.array_equal(lsg.ls_argsort(ctx, k).cpu().numpy(), np.arange(x.size))
    sp = np.array([0.0, -0.0, np.inf, -np.inf, 1e-308, -1e-308, 5e-324, -5e-324, 1.0, -1.0])
    x = np.tile(sp, 20_000)[np.random.default_rng(1).permutation(200_000)]
    k = torch.from_numpy(x.copy()).to("cuda:0")
    assert np.array_equal(lsg.ls_argsort(ctx, k).cpu().numpy(), stable_perm(x))


def test_pairs_rejects_bad_value_width(ctx):
    k = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    with pytest.raises(ValueError):
        lsg.ls_sort_pairs(ctx, k, torch.zeros(8, dtype=torch.int16, device="cuda:0"))
