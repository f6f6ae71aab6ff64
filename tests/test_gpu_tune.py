"""Autotuner: it picks parameters from its candidate lists by timing real
sorts, stores them per (key type, floor(log2 n)), and a sort run with
LS_FLAG_TUNED uses them -- with output and statistics bit-exact to the
oracle run with the same parameters (the oracle takes the tuned values as
plain inputs)."""
import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2307_08637_gb300 as lsg  # noqa: E402

FANOUTS = {256, 512, 1000, 1024, 2048}
THRESHOLDS = {1024, 2048, 4096, 8192}
RATES = {0.0025, 0.005, 0.01, 0.02}


def test_autotune_then_tuned_sort_matches_oracle(tmp_path):
    ctx = lsg.Context(0)
    x = datagen.generate("lognormal", 1 << 20, 11)
    d = torch.from_numpy(x).to("cuda:0")
    before = d.clone()
    base = lsg.ls_params_default(basecase_threshold=4096)
    tuned, rep = lsg.ls_autotune(ctx, d, base)
    torch.cuda.synchronize()
    assert torch.equal(d, before)  # the tuner sorts copies
    assert tuned.fanout in FANOUTS and tuned.basecase_threshold in THRESHOLDS and tuned.sample_rate in RATES
    assert tuned.recurse_model in (lsg.LS_RECURSE_REFINE_GLOBAL, lsg.LS_RECURSE_RETRAIN)
    assert rep.configs >= 1 + 4 + 3 + 3 + 1 - 1  # base + one sweep per parameter
    assert 0 < rep.best_ms <= rep.base_ms
    # the table holds exactly this entry
    recs = lsg.tune_text_to_json(lsg.ls_tune_export(ctx))
    assert len(recs) == 1
    r = recs[0]
    assert (r["dtype"], r["log2n"]) == (lsg.LS_F64, 20)
    assert (r["fanout"], r["basecase_threshold"], r["sample_rate"], r["recurse_model"]) == (
        tuned.fanout, tuned.basecase_threshold, tuned.sample_rate, tuned.recurse_model)
    # a sort flagged TUNED uses the entry (and sizes its workspace for it)
    p = lsg.ls_params_default(flags=lsg.LS_FLAG_TUNED)
    assert lsg.ls_workspace_size(ctx, x.size, 1, lsg.LS_F64, p) == lsg.ls_workspace_size(ctx, x.size, 1, lsg.LS_F64, tuned)
    st = lsg.ls_sort(ctx, d, p)
    got = d.cpu().numpy()
    out, rc, tr, _, _ = oracle.sort(x, oracle.params(fanout=tuned.fanout, basecase_threshold=tuned.basecase_threshold,
                                                     sample_rate=tuned.sample_rate,
                                                     recurse_model=tuned.recurse_model))
    assert rc == 0
    assert np.array_equal(got.view(np.uint64), out.view(np.uint64))
    assert st.root_decision == tr.root_decision and st.root_sample_size == tr.root_sample_size
    if st.root_decision == lsg.LS_DEC_LEARNED:
        assert st.root_nbuckets == tuned.fanout
    assert st.levels() == tr.levels()
    # JSON round trip into a fresh context reproduces the table
    path = tmp_path / "tune.json"
    lsg.save_tuning(ctx, str(path))
    ctx2 = lsg.Context(0)
    lsg.load_tuning(ctx2, str(path))
    assert lsg.tune_text_to_json(lsg.ls_tune_export(ctx2)) == recs
    ctx2.close()
    ctx.close()


def test_autotune_segmented_then_tuned_segmented_sort_matches_oracle():
    """The segmented tuner times ls_sort_segmented on the caller's batch and
    stores the winner under the mean segment length, where a segmented sort
    flagged TUNED finds it."""
    ctx = lsg.Context(0)
    keys, off, _ = datagen.segmented(96, 8, lo=1000, hi=2e5)
    d = torch.from_numpy(keys).to("cuda:0")
    before = d.clone()
    tuned, rep = lsg.ls_autotune_segmented(ctx, d, off, lsg.ls_params_default())
    torch.cuda.synchronize()
    assert torch.equal(d, before)
    assert tuned.fanout in FANOUTS and tuned.basecase_threshold in THRESHOLDS and tuned.sample_rate in RATES
    assert 0 < rep.best_ms <= rep.base_ms
    recs = lsg.tune_text_to_json(lsg.ls_tune_export(ctx))
    mean = int(off[-1]) // (off.size - 1)
    assert [(r["dtype"], r["log2n"]) for r in recs] == [(lsg.LS_F64, mean.bit_length() - 1)]
    st, dec = lsg.ls_sort_segmented(ctx, d, off, lsg.ls_params_default(flags=lsg.LS_FLAG_TUNED))
    out, rc, tr, odec = oracle.sort_segmented(keys, off, oracle.params(
        fanout=tuned.fanout, basecase_threshold=tuned.basecase_threshold, sample_rate=tuned.sample_rate,
        recurse_model=tuned.recurse_model))
    assert rc == 0
    assert np.array_equal(d.cpu().numpy().view(np.uint64), out.view(np.uint64))
    assert np.array_equal(np.asarray(dec), odec)
    assert st.levels() == tr.levels()
    with pytest.raises(ValueError):
        lsg.ls_autotune_segmented(ctx, d, np.array([0, keys.size + 1], dtype=np.uint64))
    ctx.close()


def test_tuned_flag_without_entry_uses_given_params():
    ctx = lsg.Context(0)
    x = datagen.generate("normal", 300_000, 4)
    d = torch.from_numpy(x).to("cuda:0")
    st = lsg.ls_sort(ctx, d, lsg.ls_params_default(flags=lsg.LS_FLAG_TUNED, fanout=512))
    out, rc, tr, _, _ = oracle.sort(x, oracle.params(fanout=512))
    assert rc == 0 and np.array_equal(d.cpu().numpy().view(np.uint64), out.view(np.uint64))
    assert st.levels() == tr.levels()
    ctx.close()


@pytest.mark.parametrize("bad", ["0 20 1000 4096 0.01 0\n1 2 3\n",          # short line
                                 "2 20 1000 4096 0.01 0 1.0\n",              # dtype
                                 "0 20 1 4096 0.01 0 1.0\n",                 # fanout
                                 "0 20 1000 9000 0.01 0 1.0\n",              # threshold
                                 "0 20 1000 4096 0 0 1.0\n",                 # rate
                                 "0 20 1000 4096 0.01 3 1.0\n",              # recursion
                                 "0 20 1000 4096 0.01 0 1.0 extra\n"])       # trailing text
def test_tune_import_rejects_malformed_text(bad):
    ctx = lsg.Context(0)
    with pytest.raises(lsg.LSError):
        lsg.ls_tune_import(ctx, bad)
    assert lsg.ls_tune_export(ctx) == ""  # nothing was added
    ctx.close()
