"""ls_sort_host_batch: several host arrays sorted with the copies pipelined
against the sorts; every array must come back exactly as ls_sort (and the
independent numpy order) gives it, including empty and one-key arrays, and
with both pinned and pageable host memory."""
import numpy as np
import pytest

import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2307_08637_gb300 as lsg  # noqa: E402


def ord_sorted(x):
    """Ascending order under the IEEE totalOrder map (u64: plain order)."""
    b = x.view(np.uint64)
    if x.dtype == np.float64:
        o = np.where(b >> np.uint64(63), ~b, b | np.uint64(1 << 63))
        s = np.sort(o)
        back = np.where(s >> np.uint64(63), s & np.uint64(0x7FFFFFFFFFFFFFFF), ~s)
        return back.view(np.float64)
    return np.sort(b)


@pytest.mark.parametrize("pinned", [True, False])
def test_host_batch_f64(pinned):
    ctx = lsg.Context(0)
    sizes = [0, 1, 5, 300_001, 2_000_000, 17, 1_000_000]
    dists = ["normal", "lognormal", "uniform01", "mix_gauss", "exponential", "chisquared", "uniform_1e6"]
    src = [datagen.generate(d, n, 40 + i) for i, (d, n) in enumerate(zip(dists, sizes))]
    if pinned:
        bufs = [torch.from_numpy(x.copy()).pin_memory().numpy() for x in src]
    else:
        bufs = [x.copy() for x in src]
    p = lsg.ls_params_default(basecase_threshold=4096)
    sts = lsg.ls_sort_host_batch(ctx, bufs, p, stats=True)
    assert len(sts) == len(bufs)
    for x, y, st in zip(src, bufs, sts):
        assert np.array_equal(y.view(np.uint64), ord_sorted(x).view(np.uint64))
        if x.size > 1:
            d = torch.from_numpy(x).to("cuda:0")
            st1 = lsg.ls_sort(ctx, d, p)
            assert st.levels() == st1.levels() and st.root_decision == st1.root_decision
    ctx.close()


def test_host_batch_u64_duplicates():
    ctx = lsg.Context(0)
    src = [datagen.generate(d, 400_000, 3) for d in ("zipf", "root_dups", "two_dups", "skewed_u64")]
    bufs = [torch.from_numpy(x.copy().view(np.int64)).pin_memory().numpy().view(np.uint64) for x in src]
    lsg.ls_sort_host_batch(ctx, bufs)
    for x, y in zip(src, bufs):
        assert np.array_equal(y, np.sort(x))
    ctx.close()


def test_host_batch_rejects_mixed_types():
    ctx = lsg.Context(0)
    with pytest.raises(TypeError):
        lsg.ls_sort_host_batch(ctx, [np.zeros(4), np.zeros(4, dtype=np.uint64)])
    ctx.close()
