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
