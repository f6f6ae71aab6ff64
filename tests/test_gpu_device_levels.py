"""Levels planned on the device (LS_FLAG_DEVICE_LEVELS: the device work queue
run as one CUDA graph), the same queue launched batch by batch from the host
(with pass timing), and levels planned on the host (the default): the three
forms must give
the oracle's sorted output and per-level statistics bit for bit.  The cases
cover deep refinement chains, the radix split, the depth-limit fallback,
items handed back to the host planner (buckets below a splitter tree draw
samples), several batches per level and segmented batches."""
import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2307_08637_gb300 as lsg  # noqa: E402

FORMS = {"graph": lsg.LS_FLAG_DEVICE_LEVELS, "host_iterated": lsg.LS_FLAG_DEVICE_LEVELS | lsg.LS_FLAG_TIME_PASSES,
         "host_planned": 0}
LOOPS = {"graph": (lsg.LS_LOOP_GRAPH, lsg.LS_LOOP_GRAPH_PDL), "host_iterated": (lsg.LS_LOOP_DEVICE,),
         "host_planned": (lsg.LS_LOOP_HOST,)}


def _check_form(name, st):
    assert st.level_loop in LOOPS[name], (name, st.level_loop)
    assert (st.device_batches > 0) == (name != "host_planned"), (name, st.device_batches)


@pytest.fixture(scope="module")
def ctx():
    c = lsg.Context(0)
    yield c
    c.close()


def _check(ctx, x, **kw):
    out, rc, tr, _, _ = oracle.sort(x, oracle.params(**kw))
    assert rc == 0
    for name, flag in FORMS.items():
        d = torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")
        st = lsg.ls_sort(ctx, d, lsg.ls_params_default(flags=flag, **kw))
        got = d.cpu().numpy()
        bad = np.nonzero(got.view(np.uint64) != out.view(np.uint64))[0]
        assert bad.size == 0, (name, "sorted output differs", bad[:5])
        assert st.root_decision == tr.root_decision, name
        assert st.levels() == tr.levels(), (name, st.levels(), tr.levels())
        _check_form(name, st)
    return tr


@pytest.mark.parametrize("dist", ["normal", "lognormal", "mix_gauss", "uniform_1e6"])
def test_device_levels_f64(ctx, dist):
    x = datagen.generate(dist, 1_500_000, 21)
    tr = _check(ctx, x, basecase_threshold=512)
    assert tr.levels_used >= 3


@pytest.mark.parametrize("dist", ["normal", "exponential"])
def test_device_levels_bench_parameters(ctx, dist):
    """The bench's parameters (B = 1000, T = 4096: no item of the queue
    uses the direct classifier)."""
    x = datagen.generate(dist, 6_000_000, 25)
    _check(ctx, x, basecase_threshold=4096)


def test_device_levels_deep_small_fanout(ctx):
    """Fanout 16, T = 16: about five refinement levels, several batches per
    level (more than 2048 items), refinement up to B^6."""
    x = datagen.generate("exponential", 800_000, 22)
    tr = _check(ctx, x, fanout=16, basecase_threshold=16, partitioner=oracle.PART_LEARNED)
    assert max(lv["items"] for lv in tr.levels()) > 2048


def test_device_levels_radix_and_depth_limit(ctx):
    """Clustered keys: flat model regions take the radix split; max_depth 3
    sends the rest to the fallback."""
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.standard_normal(300_000), np.full(200_000, 0.125),
                        0.125 + rng.integers(0, 64, 200_000) * 2.0**-50])
    rng.shuffle(x)
    tr = _check(ctx, x, basecase_threshold=64, partitioner=oracle.PART_LEARNED)
    assert any(lv["radix"] for lv in tr.levels())
    _check(ctx, x, basecase_threshold=64, partitioner=oracle.PART_LEARNED, max_depth=3)


@pytest.mark.parametrize("dist", ["zipf", "two_dups", "skewed_u64"])
def test_device_levels_u64_handed_back(ctx, dist):
    """Duplicate-heavy keys: splitter-tree items whose buckets draw samples
    come back to the host planner; learned descendants go to the device
    queue again."""
    x = datagen.generate(dist, 600_000, 23)
    _check(ctx, x, basecase_threshold=256)


def test_device_levels_segmented(ctx):
    keys, off, _ = datagen.segmented(300, 6, lo=100, hi=2e5)
    p_o = oracle.params(min_learned_n=20_000, basecase_threshold=256)
    out, rc, tr, dec = oracle.sort_segmented(keys, off, p_o)
    assert rc == 0
    for name, flag in FORMS.items():
        d = torch.from_numpy(keys.copy()).to("cuda:0")
        st, gdec = lsg.ls_sort_segmented(ctx, d, off, lsg.ls_params_default(flags=flag, min_learned_n=20_000,
                                                                           basecase_threshold=256))
        assert np.array_equal(d.cpu().numpy().view(np.uint64), out.view(np.uint64)), name
        assert np.array_equal(np.asarray(gdec), dec), name
        assert st.levels() == tr.levels(), name
        _check_form(name, st)


def test_device_levels_graph_reused(ctx):
    """The same array and workspace sorted again reuse the captured graph;
    a second array gets its own."""
    x = datagen.generate("chisquared", 700_000, 24)
    out, rc, tr, _, _ = oracle.sort(x, oracle.params())
    d = torch.from_numpy(x).to("cuda:0")
    ws = ctx.workspace(x.size, 1, lsg.LS_F64, lsg.ls_params_default())
    p = lsg.ls_params_default(flags=lsg.LS_FLAG_DEVICE_LEVELS)
    for _ in range(3):
        d.copy_(torch.from_numpy(x))
        st = lsg.ls_sort(ctx, d, p, workspace=ws)
        assert np.array_equal(d.cpu().numpy().view(np.uint64), out.view(np.uint64))
        assert st.levels() == tr.levels()
        _check_form("graph", st)
    e = torch.from_numpy(x).to("cuda:0")
    st = lsg.ls_sort(ctx, e, p, workspace=ws)
    assert np.array_equal(e.cpu().numpy().view(np.uint64), out.view(np.uint64))
    _check_form("graph", st)
