"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, on
the same seeded inputs.  Integer results (sorted keys, bucket ids,
histograms, decisions, per-level statistics) must be bit-exact; the FP64
model parameters must be bit-exact too because both sides evaluate the same
operations in the same order without FMA contraction."""
import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU machines but skipped there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2307_08637_gb300 as lsg  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = lsg.Context(0)
    yield c
    c.close()


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def oparams(**kw):
    return oracle.params(**kw)


def gparams(**kw):
    return lsg.ls_params_default(**kw)


def assert_model_equal(om, gm):
    od, gd = om.to_dict(), gm.to_dict()
    assert od["L"] == gd["L"]
    for k in ("xmin", "xmax", "root_x0", "root_a", "root_b"):
        assert np.float64(od[k]).view(np.uint64) == np.float64(gd[k]).view(np.uint64), (k, od[k], gd[k])
    for k in ("leaf_x0", "leaf_a", "leaf_b", "leaf_lo", "leaf_hi"):
        a, b = np.asarray(od[k]), np.asarray(gd[k])
        bad = np.nonzero(a.view(np.uint64) != b.view(np.uint64))[0]
        assert bad.size == 0, (k, bad[:5], a[bad[:5]], b[bad[:5]])
    assert np.array_equal(od["leaf_count"], gd["leaf_count"])


# ------------------------------------------------------------------ fit

@pytest.mark.parametrize("dist,n,L", [("uniform01", 2**20, 1000), ("normal", 10**6, 1000),
                                      ("lognormal", 500_000, 1024), ("mix_gauss", 400_000, 1000),
                                      ("skewed_u64", 600_000, 1000), ("uniform_1e6", 300_000, 257)])
def test_fit_parity(ctx, dist, n, L):
    x = datagen.generate(dist, n, 1)
    op = oparams(fanout=L)
    tr, om, _, osamp = oracle.root_decision(x, op)
    gm, gst, gsamp = lsg.ls_fit(ctx, to_dev(x), gparams(fanout=L), want_sample=True)
    # the same sample, sorted the same way
    assert np.array_equal(gsamp.cpu().numpy().view(np.uint64), osamp.view(np.uint64))
    assert gst.root_sample_size == tr.root_sample_size
    assert gst.root_dups == tr.root_dups
    assert gst.root_imbalance_max == tr.root_imbalance_max
    assert_model_equal(om, gm)


# ------------------------------------------------------------- classify

@pytest.mark.parametrize("mode", [lsg.LS_CLASSIFY_DIRECT, lsg.LS_CLASSIFY_DIRECTORY, lsg.LS_CLASSIFY_TREE,
                                  lsg.LS_CLASSIFY_GUESS])
@pytest.mark.parametrize("dist", ["uniform01", "normal", "exponential", "skewed_u64"])
def test_classify_parity(ctx, dist, mode):
    x = datagen.generate(dist, 300_001, 5)
    s = np.sort(x[oracle.sample_positions(17, x.size, 3000).astype(np.int64)])
    om, ok = oracle.fit(s, 1000)
    assert ok
    gm = lsg.Model.from_dict(om.to_dict())
    for k, g in ((0, 0), (1, 7), (1, 500), (2, 123456)):
        oid, oh = oracle.classify(om, x, 1000, k, g)
        gid, gh = lsg.ls_classify(ctx, gm, to_dev(x), k=k, g=g, mode=mode)
        gid = gid.cpu().numpy().view(np.uint32)
        bad = np.nonzero(gid != oid)[0]
        assert bad.size == 0, (k, g, bad[:5], gid[bad[:5]], oid[bad[:5]])
        assert np.array_equal(gh.cpu().numpy().astype(np.uint64), oh)


def test_classify_guess_on_shifted_narrow_keys(ctx):
    """Keys 1000 + 1e-3 x: the FP32 image cannot resolve them, the exact
    pivots must still give the FP64 buckets."""
    x = 1000.0 + 1e-3 * datagen.generate("normal", 200_000, 6)
    s = np.sort(x[:4000])
    om, ok = oracle.fit(s, 1000)
    gm = lsg.Model.from_dict(om.to_dict())
    for k, g in ((0, 0), (1, 433)):
        oid, oh = oracle.classify(om, x, 1000, k, g)
        gid, gh = lsg.ls_classify(ctx, gm, to_dev(x), k=k, g=g, mode=lsg.LS_CLASSIFY_GUESS)
        assert np.array_equal(gid.cpu().numpy().view(np.uint32), oid)


def test_classify_special_keys(ctx):
    """+-0, +-inf, subnormals, keys outside the sample range, u64 near 2^64."""
    s = np.sort(datagen.generate("normal", 5000, 3))
    om, _ = oracle.fit(s, 100)
    gm = lsg.Model.from_dict(om.to_dict())
    x = np.array([-np.inf, -1e308, -7.0, -0.0, 0.0, 5e-324, -5e-324, 1e-300, 3.0, 1e308, np.inf] * 3)
    for mode in (lsg.LS_CLASSIFY_DIRECT, lsg.LS_CLASSIFY_DIRECTORY, lsg.LS_CLASSIFY_TREE, lsg.LS_CLASSIFY_GUESS):
        gid, _ = lsg.ls_classify(ctx, gm, to_dev(x), mode=mode)
        oid, _ = oracle.classify(om, x, 100)
        assert np.array_equal(gid.cpu().numpy().view(np.uint32), oid)
    u = np.sort(datagen.generate("skewed_u64", 5000, 3))
    om, _ = oracle.fit(u, 64)
    gm = lsg.Model.from_dict(om.to_dict())
    y = np.array([0, 1, 2**53, 2**53 + 1, 2**63, 2**64 - 2, 2**64 - 1], dtype=np.uint64)
    for mode in (lsg.LS_CLASSIFY_DIRECT, lsg.LS_CLASSIFY_DIRECTORY, lsg.LS_CLASSIFY_GUESS):
        gid, _ = lsg.ls_classify(ctx, gm, to_dev(y), mode=mode)
        oid, _ = oracle.classify(om, y, 64)
        assert np.array_equal(gid.cpu().numpy().view(np.uint32), oid)


# ---------------------------------------------------------- full sorts

def run_both(ctx, x, **kw):
    tr_keys = {k: v for k, v in kw.items()}
    out, rc, tr, _, hist = oracle.sort(x, oparams(**tr_keys))
    assert rc == 0
    d = to_dev(x)
    st = lsg.ls_sort(ctx, d, gparams(**kw))
    got = d.cpu().numpy()
    return out, tr, hist, got, st


def assert_same_sort(out, tr, got, st):
    bad = np.nonzero(got.view(np.uint64) != out.view(np.uint64))[0]
    assert bad.size == 0, ("sorted output differs", bad[:5], got[bad[:5]], out[bad[:5]])
    assert st.root_decision == tr.root_decision
    assert st.root_sample_size == tr.root_sample_size
    assert st.root_dups == tr.root_dups
    assert st.root_imbalance_max == tr.root_imbalance_max
    gl, ol = st.levels(), tr.levels()
    assert gl == ol, ("level stats", gl, ol)


def test_sort_parity_uniform_2pow20_learned(ctx):
    """The 2^20-key U[0,1) workload: RMI B=1000 on a 1% sample, T=16, learned."""
    x = datagen.generate("uniform01", 2**20, 1)
    out, tr, hist, got, st = run_both(ctx, x, partitioner=oracle.PART_LEARNED, fanout=1000, basecase_threshold=16)
    assert tr.root_decision == oracle.DEC_LEARNED
    assert_same_sort(out, tr, got, st)


@pytest.mark.parametrize("dist", datagen.F64_DISTS)
@pytest.mark.parametrize("part", [oracle.PART_AUTO, oracle.PART_SPLITTER])
def test_sort_parity_f64_distributions(ctx, dist, part):
    x = datagen.generate(dist, 700_001, 2)
    out, tr, hist, got, st = run_both(ctx, x, partitioner=part)
    assert_same_sort(out, tr, got, st)


@pytest.mark.parametrize("dist", ["zipf", "root_dups", "two_dups", "skewed_u64"])
def test_sort_parity_u64_duplicates(ctx, dist):
    x = datagen.generate(dist, 500_000, 3)
    out, tr, hist, got, st = run_both(ctx, x)
    assert_same_sort(out, tr, got, st)


@pytest.mark.parametrize("kw", [dict(recurse_model=oracle.RECURSE_RETRAIN, min_learned_n=20_000),
                                dict(basecase_threshold=1024, fanout=256),
                                dict(basecase_threshold=4096, fanout=4096, splitter_fanout=2048),
                                dict(partitioner=oracle.PART_LEARNED, fanout=2, basecase_threshold=16),
                                dict(max_depth=1, basecase_threshold=16),
                                dict(sample_rate=1.0, partitioner=oracle.PART_LEARNED),
                                dict(classify_mode=3), dict(classify_mode=1), dict(classify_mode=2),
                                dict(classify_mode=4)])
def test_sort_parity_options(ctx, kw):
    x = datagen.generate("mix_gauss", 300_000, 4)
    okw = {k: v for k, v in kw.items() if k != "classify_mode"}
    out, rc, tr, _, _ = oracle.sort(x, oparams(**okw))
    d = to_dev(x)
    st = lsg.ls_sort(ctx, d, gparams(**kw))
    assert_same_sort(out, tr, d.cpu().numpy(), st)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 15, 16, 17, 255, 256, 257, 4095, 4096, 4097, 100_003])
def test_sort_edge_sizes(ctx, n):
    x = datagen.generate("normal", n, 9)
    out, tr, hist, got, st = run_both(ctx, x)
    assert_same_sort(out, tr, got, st)


def _large_span_inputs():
    """Single spans of 257..8192 keys (the root goes straight to the block
    base case): spread keys, keys sharing their high word, clustered keys
    (one slot overflows and the block falls back to the bitonic network),
    two values, and all-equal-but-one."""
    rng = np.random.default_rng(11)
    cases = []
    for n in (257, 300, 1000, 2049, 4000, 4096):
        cases.append(("normal", n, rng.standard_normal(n)))
        cases.append(("low_word", n, rng.integers(0, 5000, n, dtype=np.uint64)))
        c = np.full(n, 7.25)
        c[rng.permutation(n)[: n // 10]] = rng.standard_normal(n // 10)
        cases.append(("clustered", n, c))
        cases.append(("two_values", n, np.where(rng.random(n) < 0.5, -3.0, 3.0)))
        e = np.full(n, 1.5)
        e[rng.integers(0, n)] = -2.0
        cases.append(("one_differs", n, e))
    for n in (4097, 6000, 8192):
        cases.append(("normal", n, rng.standard_normal(n)))
    return cases


@pytest.mark.parametrize("name,n,x", _large_span_inputs(), ids=lambda v: str(v) if not hasattr(v, "shape") else "")
def test_base_case_large_spans(ctx, name, n, x):
    out, tr, hist, got, st = run_both(ctx, x, basecase_threshold=8192)
    assert_same_sort(out, tr, got, st)


def test_sort_special_values_and_all_equal(ctx):
    rng = np.random.default_rng(0)
    pool = np.array([-np.inf, -1e300, -1.0, -5e-324, -0.0, 0.0, 5e-324, 0.5, 1.0, 1e300, np.inf])
    x = pool[rng.integers(0, pool.size, 200_000)]
    out, tr, hist, got, st = run_both(ctx, x)
    assert_same_sort(out, tr, got, st)
    y = np.full(150_000, 2.5)
    out, tr, hist, got, st = run_both(ctx, y)
    assert tr.root_decision == oracle.DEC_HOMOGENEOUS
    assert_same_sort(out, tr, got, st)
    u = rng.integers(0, 2**64 - 1, 200_000, dtype=np.uint64, endpoint=True)
    u[::7] = np.uint64(2**64 - 1)
    out, tr, hist, got, st = run_both(ctx, u)
    assert_same_sort(out, tr, got, st)


def test_nan_is_reported(ctx):
    x = datagen.generate("normal", 300_000, 1)
    x[123_456] = np.nan
    d = to_dev(x)
    st = lsg.ls_sort(ctx, d, gparams(), check=False)
    assert st.status == lsg.LS_ENAN


def test_segmented_parity(ctx):
    keys, off, names = datagen.segmented(64, 4, lo=100, hi=3e5)
    p_o = oparams(min_learned_n=50_000)
    out, rc, tr, dec = oracle.sort_segmented(keys, off, p_o)
    assert rc == 0
    d = to_dev(keys)
    st, gdec = lsg.ls_sort_segmented(ctx, d, off, gparams(min_learned_n=50_000))
    got = d.cpu().numpy()
    assert np.array_equal(got.view(np.uint64), out.view(np.uint64))
    assert np.array_equal(gdec, dec)
    assert st.levels() == tr.levels()


# -------------------------------------------------------- fwd / bwd

def test_fit_grad_parity(ctx):
    S = 20_000
    s = np.sort(datagen.generate("chisquared", S, 21))
    om, ok = oracle.fit(s, 64)
    d = om.to_dict()
    rng = np.random.default_rng(1)
    d["leaf_a"] = d["leaf_a"] * (1 + 0.2 * rng.standard_normal(64))
    d["leaf_b"] = d["leaf_b"] + 0.001 * rng.standard_normal(64)
    for dd in (om.to_dict(), d):
        m_o = oracle.Model.from_dict(dd)
        ga, gb, gr = oracle.fit_backward(m_o, s)
        pred, resid = oracle.fit_forward(m_o, s)
        out = lsg.ls_fit_grad(ctx, lsg.Model.from_dict(dd), to_dev(s))
        assert np.array_equal(out["grad_a"].cpu().numpy().view(np.uint64), ga.view(np.uint64))
        assert np.array_equal(out["grad_b"].cpu().numpy().view(np.uint64), gb.view(np.uint64))
        assert np.array_equal(out["grad_root"].cpu().numpy().view(np.uint64), gr.view(np.uint64))
        assert np.array_equal(out["pred"].cpu().numpy().view(np.uint64), pred.view(np.uint64))
        assert np.array_equal(out["resid"].cpu().numpy().view(np.uint64), resid.view(np.uint64))
