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


MODES = [lsg.LS_CLASSIFY_AUTO, lsg.LS_CLASSIFY_DIRECTORY, lsg.LS_CLASSIFY_TREE, lsg.LS_CLASSIFY_DIRECT,
         lsg.LS_CLASSIFY_GUESS]


@pytest.mark.parametrize("mode", MODES)
def test_static_matches_ls_classify_twice(mode):
    ctx = lsg.Context(0)
    cases = [("normal", 400_000, 1000, 3, 0, 0), ("lognormal", 300_001, 4096, 5, 1, 77),
             ("skewed_u64", 250_000, 777, 9, 0, 0)]
    for dist, n, L, seed, k, g in cases:  # calls in a row, different models
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
    hist = torch.empty(lsg.LS_MAX_FANOUT + 1, dtype=torch.int64, device="cuda:0")
    with pytest.raises(lsg.LSError):  # more leaves than LS_MAX_FANOUT: the C side rejects it
        lsg.ls_classify_static(m, d, ids, hist)
    m.L = 1000
    with pytest.raises(lsg.LSError):  # B^(k+1) past the FP64 refinement limit
        lsg.ls_classify_static(m, d, ids, hist, k=9)


def test_static_allocates_nothing():
    """The defining property: after one warm-up call per mode (which loads the
    kernels), further calls change neither torch's allocator nor the device's
    free memory."""
    m, d = _model("normal", 200_000, 1000, 4)
    ids = torch.empty(d.numel(), dtype=torch.int32, device="cuda:0")
    hist = torch.empty(1000, dtype=torch.int64, device="cuda:0")
    for mode in MODES:
        lsg.ls_classify_static(m, d, ids, hist, mode=mode)
    torch.cuda.synchronize()
    before = (torch.cuda.memory_allocated(0), torch.cuda.memory_reserved(0), torch.cuda.mem_get_info(0)[0])
    for _ in range(3):
        for mode in MODES:
            lsg.ls_classify_static(m, d, ids, hist, k=1, g=5, mode=mode)
    torch.cuda.synchronize()
    after = (torch.cuda.memory_allocated(0), torch.cuda.memory_reserved(0), torch.cuda.mem_get_info(0)[0])
    assert after == before


def test_static_rejects_bad_tensors_on_the_host():
    m, d = _model("normal", 150_000, 1000, 6)
    n = d.numel()
    ok_ids = torch.empty(n, dtype=torch.int32, device="cuda:0")
    ok_hist = torch.empty(1000, dtype=torch.int64, device="cuda:0")
    bad = [
        (d, ok_ids, torch.empty(999, dtype=torch.int64, device="cuda:0")),   # short histogram
        (d, torch.empty(n - 1, dtype=torch.int32, device="cuda:0"), ok_hist),  # short ids
        (d, ok_ids.to(torch.int64), ok_hist),                                 # wrong ids dtype
        (d, ok_ids, ok_hist.to(torch.int32)),                                 # wrong histogram dtype
        (d.cpu(), ok_ids, ok_hist),                                           # keys not on the GPU
        (d, ok_ids.cpu(), ok_hist),                                           # ids not on the keys' device
        (d[::2], ok_ids, ok_hist),                                            # strided keys
    ]
    for keys, ids, hist in bad:
        with pytest.raises(ValueError):
            lsg.ls_classify_static(m, keys, ids, hist)
    with pytest.raises(TypeError):
        lsg.ls_classify_static(m, d.to(torch.float32), ok_ids, ok_hist)
    for k in (50, 2**32 - 1, 2**32 - 2):  # past the refinement limit; k + 1 would wrap at 2^32 - 1
        with pytest.raises(lsg.LSError):
            lsg.ls_classify_static(m, d, ok_ids, ok_hist, k=k)
    with pytest.raises(lsg.LSError):
        lsg.ls_classify_static(m, d, ok_ids, ok_hist, mode=5)
