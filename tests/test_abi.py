"""The C-ABI library builds, loads and exports every symbol include/ls.h
declares; host-side argument checks work without a GPU (no compute calls)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ls.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ls_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2307_08637_gb300 as lsg

    L = lsg.lib()
    declared = _declared()
    assert set(declared) == set(lsg.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name


def test_params_default_and_host_validation():
    import paper_2307_08637_gb300 as lsg

    p = lsg.ls_params_default()
    assert (p.fanout, p.splitter_fanout, p.basecase_threshold, p.max_depth) == (1000, 1024, 16, 16)
    assert p.sample_rate == 0.01 and p.dup_frac == 0.10 and p.min_learned_n == 100000
    n = C.c_size_t()
    L = lsg.lib()
    assert L.ls_workspace_size(None, 10**6, 1, 0, C.byref(p), C.byref(n)) == lsg.LS_OK
    assert n.value > 8 * 10**6  # holds at least the ping-pong buffer
    bad = lsg.ls_params_default(fanout=1)
    assert L.ls_workspace_size(None, 10, 1, 0, C.byref(bad), C.byref(n)) == lsg.LS_EINVAL
    bad = lsg.ls_params_default(basecase_threshold=100000)
    assert L.ls_workspace_size(None, 10, 1, 0, C.byref(bad), C.byref(n)) == lsg.LS_EINVAL
    assert L.ls_workspace_size(None, 10, 1, 7, C.byref(p), C.byref(n)) == lsg.LS_EINVAL
    assert lsg.status_string(lsg.LS_ENAN) == "NaN key"


def test_model_export_import_roundtrip_and_checksum():
    import numpy as np

    import paper_2307_08637_gb300 as lsg

    m = lsg.Model()
    m.L = 7
    m.root_a = 0.125
    np.ctypeslib.as_array(m.leaf_b)[:7] = np.arange(7) / 7.0
    blob = lsg.ls_model_export(m)
    m2 = lsg.ls_model_import(blob)
    assert bytes(m2) == bytes(m)
    bad = bytearray(blob)
    bad[40] ^= 1
    with pytest.raises(lsg.LSError):
        lsg.ls_model_import(bytes(bad))


def test_oracle_and_product_share_no_code():
    """The product sources neither import nor include the oracle, and the
    oracle includes nothing of the product."""
    pkg = os.path.join(ROOT, "paper_2307_08637_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".cu", ".cuh", ".h", ".py")):
                s = open(os.path.join(dp, f)).read()
                for bad in ("import oracle", "from oracle", "ls_oracle", "lsref_"):
                    assert bad not in s, (f, bad)
    o = open(os.path.join(ROOT, "oracle", "ls_oracle.c")).read() + open(os.path.join(ROOT, "oracle", "ls_oracle.h")).read()
    for bad in ("paper_2307_08637_gb300", "ls_common", "ls_kernels", "include/ls.h"):
        assert bad not in o, bad


def test_tuning_table_text_json_roundtrip():
    """The autotuner's table format: ls_tune_export text <-> JSON records
    (pure host code; the GPU tests cover the C side)."""
    import paper_2307_08637_gb300 as lsg
    text = "0 20 1000 4096 0.01 0 3.250000\n1 26 512 2048 0.0050000000000000001 1 41.500000\n"
    recs = lsg.tune_text_to_json(text)
    assert recs == [
        {"dtype": 0, "log2n": 20, "fanout": 1000, "basecase_threshold": 4096, "sample_rate": 0.01,
         "recurse_model": 0, "ms": 3.25},
        {"dtype": 1, "log2n": 26, "fanout": 512, "basecase_threshold": 2048, "sample_rate": 0.005,
         "recurse_model": 1, "ms": 41.5}]
    assert lsg.tune_text_to_json(lsg.tune_json_to_text(recs)) == recs
    with pytest.raises(ValueError):
        lsg.tune_text_to_json("0 20 1000\n")
