"""Parity at the workloads' full sizes, in the configuration bench.py times
(fanout 1000, 1 % sample, base-case threshold 4096, Alg. 5 AUTO):

* every 1e8-key float64 distribution and every 1e8-key duplicate-heavy u64
  input: the whole sorted output against an independent sort of the same
  bytes (the sorted order under ord is unique, so torch.sort of the ord
  image must give it bit for bit);
* for several of them, the oracle's full run as well: sorted output and the
  per-level statistics (decisions, bucket fills, base-case counts);
* the 2e9-key skewed u64 workload (RETRAIN recursion): the sorted output
  against the independent sort, and the root model against the oracle's on
  the same bytes;
* the 4096-segment float64 batch (6.3e8 keys): every segment against
  independent stable sorts, per-segment root decisions against the oracle's.
"""
import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2307_08637_gb300 as lsg  # noqa: E402

N = 10**8
T = 4096
MIN64 = -(1 << 63)


def ord_signed(t, dt):
    """int64 tensor whose signed order is the keys' ord order (an involution)."""
    if dt == lsg.LS_F64:
        return t ^ ((t >> 63) & 0x7FFFFFFFFFFFFFFF)
    return t ^ MIN64


def independent_sort(bits, dt):
    """The unique ascending order of the keys, from torch.sort of their ord image."""
    s = torch.sort(ord_signed(bits, dt))[0]
    return ord_signed(s, dt)


@pytest.fixture(scope="module")
def ctx():
    c = lsg.Context(0)
    yield c
    c.close()


def run_full(ctx, x, p, oracle_trace):
    dt = lsg.LS_F64 if x.dtype == np.float64 else lsg.LS_U64
    d = torch.from_numpy(x).to("cuda:0")
    st = lsg.ls_sort(ctx, d, p)
    got = d.view(torch.int64)
    want = independent_sort(torch.from_numpy(x.view(np.int64)).to("cuda:0"), dt)
    assert torch.equal(got, want), "sorted output differs from the independent sort"
    if oracle_trace:
        kw = dict(basecase_threshold=p.basecase_threshold, fanout=p.fanout, recurse_model=p.recurse_model)
        out, rc, tr, _, _ = oracle.sort(x, oracle.params(**kw))
        assert rc == 0
        assert np.array_equal(got.cpu().numpy(), out.view(np.int64))
        assert st.root_decision == tr.root_decision
        assert st.root_sample_size == tr.root_sample_size and st.root_dups == tr.root_dups
        assert st.levels() == tr.levels()
    return st


@pytest.mark.parametrize("dist", datagen.F64_DISTS)
def test_full_1e8_f64(ctx, dist):
    x = datagen.generate(dist, N, 2)
    run_full(ctx, x, lsg.ls_params_default(basecase_threshold=T), oracle_trace=dist in ("normal", "mix_gauss"))


@pytest.mark.parametrize("dist", ["zipf", "root_dups", "two_dups"])
def test_full_1e8_u64_duplicates(ctx, dist):
    x = datagen.generate(dist, N, 3)
    run_full(ctx, x, lsg.ls_params_default(basecase_threshold=T), oracle_trace=True)


def test_full_2e9_u64_skewed_retrain(ctx):
    n = 2 * 10**9
    bits = datagen.skewed_u64_device(n, 5, "cuda:0")
    p = lsg.ls_params_default(basecase_threshold=T, recurse_model=lsg.LS_RECURSE_RETRAIN)
    # root model: the device fit against the oracle's on the same bytes
    host = bits.cpu().numpy().view(np.uint64)
    tr, om, _, _ = oracle.root_decision(host, oracle.params(basecase_threshold=T,
                                                            recurse_model=lsg.LS_RECURSE_RETRAIN))
    gm, gst, _ = lsg.ls_fit(ctx, bits.view(torch.int64), p)
    assert gst.root_sample_size == tr.root_sample_size == 2 * 10**7
    assert gst.root_dups == tr.root_dups and gst.root_imbalance_max == tr.root_imbalance_max
    od, gd = om.to_dict(), gm.to_dict()
    for k in ("xmin", "xmax", "root_x0", "root_a", "root_b"):
        assert np.float64(od[k]).view(np.uint64) == np.float64(gd[k]).view(np.uint64), k
    for k in ("leaf_x0", "leaf_a", "leaf_b", "leaf_lo", "leaf_hi"):
        assert np.array_equal(np.asarray(od[k]).view(np.uint64), np.asarray(gd[k]).view(np.uint64)), k
    del host
    # the whole sort against the independent sort
    work = bits.clone()
    st = lsg.ls_sort(ctx, work, p)
    assert st.root_decision == tr.root_decision
    ctx.free_workspace()
    want = independent_sort(bits, lsg.LS_U64)
    assert torch.equal(work, want)


def test_full_c4_segmented_4096(ctx):
    """4096 float64 segments (6.3e8 keys): every segment sorted exactly
    (independent stable sorts: by ord, then by segment), and the per-segment
    root decisions equal to the oracle's on a sample of segments."""
    keys, off, names = datagen.segmented(4096, 4)
    p = lsg.ls_params_default(basecase_threshold=T)
    d = torch.from_numpy(keys).to("cuda:0")
    st, dec = lsg.ls_sort_segmented(ctx, d, off, p)
    got = d.view(torch.int64)
    ctx.free_workspace()
    bits = torch.from_numpy(keys.view(np.int64)).to("cuda:0")
    lens = torch.from_numpy(np.diff(off).astype(np.int64)).to("cuda:0")
    seg = torch.repeat_interleave(torch.arange(lens.numel(), device="cuda:0"), lens)
    o = ord_signed(bits, lsg.LS_F64)
    o, perm = torch.sort(o, stable=True)
    seg = seg[perm]
    del perm
    seg, perm = torch.sort(seg, stable=True)
    want = ord_signed(o[perm], lsg.LS_F64)
    del o, perm, seg
    assert torch.equal(got, want)
    op = oracle.params(basecase_threshold=T)
    for s in range(0, 4096, 128):
        x = keys[int(off[s]):int(off[s + 1])]
        if x.size <= T:
            continue
        tr, _, _, _ = oracle.root_decision(x, op, segment=s)
        assert dec[s] == tr.root_decision, s
