"""ls_classify_static: the classification entry point that allocates no
device memory, for callers whose memory pool owns the device or that must
not risk cudaMalloc's synchronisation.  Its ids and histogram must equal
those of ls_classify (integers: exactly) on two calls in a row, where the
second call reuses the shared static scratch the first one left behind.

This file is named so pytest collects it last."""
import numpy as np
import pytest

import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2307_08637_gb300 as lsg  # noqa: E402


def _model(dist, n, L, seed):
    """Train a model with ls_fit (through the C ABI) on seeded keys."""
    ctx = lsg.Context(0)
    x = datagen.generate(dist, n, seed)
    d = torch.from_numpy(x).to("cuda:0")
    m, _, _ = lsg.ls_fit(ctx, d, lsg.ls_params_default(fanout=L, partitioner=lsg.LS_PART_LEARNED))
    ctx.close()
    return m, d


@pytest.mark.parametrize("mode", [lsg.LS_CLASSIFY_DIRECTORY, lsg.LS_CLASSIFY_TREE, lsg.LS_CLASSIFY_DIRECT])
def test_static_matches_ls_classify_twice(mode):
    ctx = lsg.Context(0)
    cases = [("normal", 400_000, 1000, 3, 0, 0), ("lognormal", 300_001, 4096, 5, 1, 77)]
    for dist, n, L, seed, k, g in cases:  # two calls in a row, different models
        m, d = _model(dist, n, L, seed)
        ids_ref, hist_ref = lsg.ls_classify(ctx, m, d, k=k, g=g, mode=mode)
        ids = torch.full((n,), -1, dtype=torch.int32, device="cuda:0")
        hist = torch.full((L,), -1, dtype=torch.int64, device="cuda:0")
        lsg.ls_classify_static(m, d, ids, hist, k=k, g=g, mode=mode)
        torch.cuda.synchronize()
        assert torch.equal(ids, ids_ref), (dist, mode)
        assert torch.equal(hist, hist_ref), (dist, mode)
        assert int(hist.sum()) == n
    ctx.close()


def test_static_rejects_bad_arguments():
    m = lsg.Model()
    m.L = lsg.LS_MAX_FANOUT + 1
    d = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    ids = torch.empty(4, dtype=torch.int32, device="cuda:0")
    hist = torch.empty(8, dtype=torch.int64, device="cuda:0")
    with pytest.raises(lsg.LSError):
        lsg.ls_classify_static(m, d, ids, hist)
    m.L = 1000
    with pytest.raises(lsg.LSError):  # B^(k+1) past the FP64 refinement limit
        lsg.ls_classify_static(m, d, ids, hist, k=9)
