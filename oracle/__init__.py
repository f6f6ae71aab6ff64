"""Python binding of the CPU oracle (``ls_oracle.c``).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, the smoke check in
``__graft_entry__.py`` and the cpu_baseline / reference leg of ``bench.py``
may import this package.  It shares nothing with the CUDA library in
``paper_2307_08637_gb300`` except the seeded input generators of ``datagen``.

The oracle is a plain single-threaded C implementation of LearnedSort as
described in arxiv 2307.08637: the two-layer linear RMI of Sec. 2.1 trained
on a sorted 1% sample (Sec. 2.2), made monotone (Sec. 4), the bucket
b(x) = floor(B F(x)), the splitter-tree SampleSort classifier with equality
buckets (Sec. 2.4), Alg. 5's model choice, recursion, the homogeneity check
and a base case.  Parity status of each function is given in its docstring.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ls_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblsoracle.so")
_lock = threading.Lock()
_lib = None

F64 = 0
U64 = 1
PART_AUTO, PART_LEARNED, PART_SPLITTER = 0, 1, 2
RECURSE_REFINE_GLOBAL, RECURSE_RETRAIN = 0, 1
DEC_NONE, DEC_LEARNED, DEC_SPLITTER, DEC_SPLITTER_EQ, DEC_HOMOGENEOUS, DEC_RADIX = 0, 1, 2, 3, 4, 5
MAX_FANOUT = 4096
MAX_LEVELS = 48
OK, EINVAL, ENOMEM, ENAN = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile ls_oracle.c into liblsoracle.so (gcc, -ffp-contract=off)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [
        ("fanout", C.c_uint32),
        ("splitter_fanout", C.c_uint32),
        ("basecase_threshold", C.c_uint32),
        ("max_depth", C.c_uint32),
        ("min_sample", C.c_uint32),
        ("auto_splitter_fanout", C.c_uint32),
        ("sample_rate", C.c_double),
        ("dup_frac", C.c_double),
        ("imbalance_tau", C.c_double),
        ("min_learned_n", C.c_uint64),
        ("seed", C.c_uint64),
        ("partitioner", C.c_int32),
        ("recurse_model", C.c_int32),
    ]


class Model(C.Structure):
    _fields_ = [
        ("L", C.c_uint32),
        ("S", C.c_uint32),
        ("xmin", C.c_double),
        ("xmax", C.c_double),
        ("root_x0", C.c_double),
        ("root_a", C.c_double),
        ("root_b", C.c_double),
        ("leaf_x0", C.c_double * MAX_FANOUT),
        ("leaf_a", C.c_double * MAX_FANOUT),
        ("leaf_b", C.c_double * MAX_FANOUT),
        ("leaf_lo", C.c_double * MAX_FANOUT),
        ("leaf_hi", C.c_double * MAX_FANOUT),
        ("leaf_count", C.c_uint32 * MAX_FANOUT),
    ]

    def to_dict(self) -> dict:
        L = self.L
        g = lambda f: np.ctypeslib.as_array(getattr(self, f))[:L].copy()
        return {
            "L": L, "S": self.S, "xmin": self.xmin, "xmax": self.xmax,
            "root_x0": self.root_x0, "root_a": self.root_a, "root_b": self.root_b,
            "leaf_x0": g("leaf_x0"), "leaf_a": g("leaf_a"), "leaf_b": g("leaf_b"),
            "leaf_lo": g("leaf_lo"), "leaf_hi": g("leaf_hi"), "leaf_count": g("leaf_count"),
        }

    @classmethod
    def from_dict(cls, d: dict) -> "Model":
        m = cls()
        L = int(d["L"])
        m.L = L
        m.S = int(d.get("S", 0))
        for k in ("xmin", "xmax", "root_x0", "root_a", "root_b"):
            setattr(m, k, float(d[k]))
        for k in ("leaf_x0", "leaf_a", "leaf_b", "leaf_lo", "leaf_hi"):
            np.ctypeslib.as_array(getattr(m, k))[:L] = np.asarray(d[k], dtype=np.float64)
        if "leaf_count" in d:
            np.ctypeslib.as_array(m.leaf_count)[:L] = np.asarray(d["leaf_count"], dtype=np.uint32)
        return m


class Splitter(C.Structure):
    _fields_ = [
        ("nsplit", C.c_uint32),
        ("nbuckets", C.c_uint32),
        ("equality", C.c_int32),
        ("split", C.c_uint64 * MAX_FANOUT),
    ]


class LevelStats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in (
        "items", "learned", "splitter", "splitter_eq", "homogeneous", "noprogress", "base_items",
        "base_keys", "fallback_items", "fallback_keys", "keys", "max_child", "sumsq_child", "eq_keys", "radix")]


class Trace(C.Structure):
    _fields_ = [
        ("status", C.c_int32),
        ("root_decision", C.c_int32),
        ("root_sample_size", C.c_uint64),
        ("root_dups", C.c_uint64),
        ("root_imbalance_max", C.c_uint64),
        ("root_nbuckets", C.c_uint32),
        ("levels_used", C.c_uint32),
        ("level", LevelStats * MAX_LEVELS),
    ]

    def levels(self) -> list[dict]:
        out = []
        for i in range(self.levels_used):
            ls = self.level[i]
            out.append({n: int(getattr(ls, n)) for n, _ in LevelStats._fields_})
        return out


_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.lsref_ord.restype = C.c_uint64
            L.lsref_ord.argtypes = [C.c_uint64, C.c_int]
            L.lsref_unord.restype = C.c_uint64
            L.lsref_unord.argtypes = [C.c_uint64, C.c_int]
            L.lsref_key_value.restype = C.c_double
            L.lsref_key_value.argtypes = [C.c_uint64, C.c_int]
            L.lsref_splitmix64.restype = C.c_uint64
            L.lsref_splitmix64.argtypes = [C.c_uint64]
            L.lsref_seed_item.restype = C.c_uint64
            L.lsref_seed_item.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint64]
            L.lsref_sample_size.restype = C.c_uint64
            L.lsref_sample_size.argtypes = [C.c_uint64, C.POINTER(Params)]
            L.lsref_sample_positions.restype = None
            L.lsref_sample_positions.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64, _u64p]
            L.lsref_params_default.argtypes = [C.POINTER(Params)]
            L.lsref_fit.restype = C.c_int
            L.lsref_fit.argtypes = [_u64p, C.c_uint64, C.c_int, C.c_uint32, C.POINTER(Model)]
            L.lsref_model_F.restype = C.c_double
            L.lsref_model_F.argtypes = [C.POINTER(Model), C.c_double]
            L.lsref_model_leaf.restype = C.c_uint32
            L.lsref_model_leaf.argtypes = [C.POINTER(Model), C.c_double]
            L.lsref_refine_id.restype = C.c_uint32
            L.lsref_refine_id.argtypes = [C.POINTER(Model), C.c_uint64, C.c_int, C.c_uint32, C.c_uint32,
                                          C.c_uint64]
            L.lsref_classify.restype = None
            L.lsref_classify.argtypes = [C.POINTER(Model), _u64p, C.c_uint64, C.c_int, C.c_uint32, C.c_uint32,
                                         C.c_uint64, _u32p, _u64p]
            L.lsref_fit_forward.restype = None
            L.lsref_fit_forward.argtypes = [C.POINTER(Model), _u64p, C.c_uint64, C.c_int, _f64p, _f64p]
            L.lsref_fit_backward.restype = None
            L.lsref_fit_backward.argtypes = [C.POINTER(Model), _u64p, C.c_uint64, C.c_int, _f64p, _f64p,
                                             _f64p]
            L.lsref_splitter_build.restype = None
            L.lsref_splitter_build.argtypes = [_u64p, C.c_uint64, C.c_int, C.c_uint32, C.c_int,
                                               C.POINTER(Splitter)]
            L.lsref_splitter_bucket.restype = C.c_uint32
            L.lsref_splitter_bucket.argtypes = [C.POINTER(Splitter), C.c_uint64]
            L.lsref_splitter_classify.restype = None
            L.lsref_splitter_classify.argtypes = [C.POINTER(Splitter), _u64p, C.c_uint64, C.c_int, _u32p, _u64p]
            L.lsref_sort.restype = C.c_int
            L.lsref_sort.argtypes = [_u64p, C.c_uint64, C.c_int, C.POINTER(Params), C.POINTER(Trace),
                                     C.c_void_p, C.c_void_p]
            L.lsref_sort_segmented.restype = C.c_int
            L.lsref_sort_segmented.argtypes = [_u64p, _u64p, C.c_uint32, C.c_int, C.POINTER(Params),
                                               C.POINTER(Trace), C.c_void_p]
            L.lsref_root_decision.restype = C.c_int
            L.lsref_root_decision.argtypes = [_u64p, C.c_uint64, C.c_int, C.POINTER(Params), C.c_uint64,
                                              C.POINTER(Trace), C.POINTER(Model), C.POINTER(Splitter), C.c_void_p]
            for fn in ("lsref_sizeof_model", "lsref_sizeof_trace", "lsref_sizeof_params", "lsref_sizeof_splitter"):
                getattr(L, fn).restype = C.c_size_t
                getattr(L, fn).argtypes = []
            assert L.lsref_sizeof_model() == C.sizeof(Model)
            assert L.lsref_sizeof_trace() == C.sizeof(Trace)
            assert L.lsref_sizeof_params() == C.sizeof(Params)
            assert L.lsref_sizeof_splitter() == C.sizeof(Splitter)
            _lib = L
    return _lib


# ----------------------------------------------------------------- helpers

def as_bits(keys: np.ndarray) -> tuple[np.ndarray, int]:
    """(uint64 bit patterns, dtype code) of a float64 or uint64 key array."""
    keys = np.ascontiguousarray(keys)
    if keys.dtype == np.float64:
        return keys.view(np.uint64), F64
    if keys.dtype == np.uint64:
        return keys, U64
    raise TypeError(f"keys must be float64 or uint64, got {keys.dtype}")


def params(**kw) -> Params:
    p = Params()
    lib().lsref_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def key_value(bits: int, dtype: int) -> float:
    """The value the model reads for one key (Sec. 2.1's x): the double
    itself, or a u64 converted to the nearest double (ties to even)."""
    return float(lib().lsref_key_value(bits, dtype))


def ord_keys(keys: np.ndarray) -> np.ndarray:
    bits, dt = as_bits(keys)
    L = lib()
    return np.fromiter((L.lsref_ord(int(b), dt) for b in bits), dtype=np.uint64, count=bits.size)


def sample_positions(seed_item: int, n: int, S: int) -> np.ndarray:
    out = np.zeros(max(S, 1), dtype=np.uint64)
    lib().lsref_sample_positions(seed_item, n, S, out)
    return out[:S]


def seed_item(seed: int, segment: int, level: int, gidx: int) -> int:
    return int(lib().lsref_seed_item(seed, segment, level, gidx))


def sample_size(n: int, p: Params) -> int:
    return int(lib().lsref_sample_size(n, C.byref(p)))


def fit(sorted_sample: np.ndarray, L: int) -> tuple[Model, bool]:
    """Fit the two-layer RMI on a sample already sorted by ord."""
    bits, dt = as_bits(sorted_sample)
    m = Model()
    ok = lib().lsref_fit(np.ascontiguousarray(bits), bits.size, dt, L, C.byref(m))
    return m, bool(ok == 1)


def model_F(m: Model, x: float) -> float:
    return float(lib().lsref_model_F(C.byref(m), float(x)))


def classify(m: Model, keys: np.ndarray, B: int, k: int = 0, g: int = 0) -> tuple[np.ndarray, np.ndarray]:
    bits, dt = as_bits(keys)
    ids = np.zeros(max(bits.size, 1), dtype=np.uint32)
    hist = np.zeros(B, dtype=np.uint64)
    lib().lsref_classify(C.byref(m), np.ascontiguousarray(bits), bits.size, dt, B, k, g, ids, hist)
    return ids[:bits.size], hist


def fit_forward(m: Model, sorted_sample: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    bits, dt = as_bits(sorted_sample)
    pred = np.zeros(max(bits.size, 1))
    resid = np.zeros(max(bits.size, 1))
    lib().lsref_fit_forward(C.byref(m), np.ascontiguousarray(bits), bits.size, dt, pred, resid)
    return pred[:bits.size], resid[:bits.size]


def fit_backward(m: Model, sorted_sample: np.ndarray) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    bits, dt = as_bits(sorted_sample)
    ga = np.zeros(m.L)
    gb = np.zeros(m.L)
    gr = np.zeros(2)
    lib().lsref_fit_backward(C.byref(m), np.ascontiguousarray(bits), bits.size, dt, ga, gb, gr)
    return ga, gb, gr


def splitter_build(sorted_sample: np.ndarray, bs_max: int, force_equality: bool = False) -> Splitter:
    bits, dt = as_bits(sorted_sample)
    t = Splitter()
    lib().lsref_splitter_build(np.ascontiguousarray(bits), bits.size, dt, bs_max, int(force_equality), C.byref(t))
    return t


def splitter_classify(t: Splitter, keys: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    bits, dt = as_bits(keys)
    ids = np.zeros(max(bits.size, 1), dtype=np.uint32)
    hist = np.zeros(max(t.nbuckets, 1), dtype=np.uint64)
    lib().lsref_splitter_classify(C.byref(t), np.ascontiguousarray(bits), bits.size, dt, ids, hist)
    return ids[:bits.size], hist[:t.nbuckets]


def sort(keys: np.ndarray, p: Params | None = None, want_model: bool = False):
    """Sort a copy of ``keys``; returns (sorted, status, trace, model|None, root_hist)."""
    p = p or params()
    out = np.array(keys, copy=True)
    bits, dt = as_bits(out)
    tr = Trace()
    m = Model()
    hist = np.zeros(2 * MAX_FANOUT + 2, dtype=np.uint64)
    rc = lib().lsref_sort(bits, bits.size, dt, C.byref(p), C.byref(tr), C.addressof(m),
                          hist.ctypes.data)
    nb = tr.root_nbuckets
    return out, int(rc), tr, (m if want_model else None), hist[:nb].copy()


def sort_segmented(keys: np.ndarray, offsets: np.ndarray, p: Params | None = None):
    """Sort each [off[s], off[s+1]) independently; returns (sorted, status, trace, decisions)."""
    p = p or params()
    out = np.array(keys, copy=True)
    bits, dt = as_bits(out)
    off = np.ascontiguousarray(offsets, dtype=np.uint64)
    nseg = off.size - 1
    dec = np.zeros(max(nseg, 1), dtype=np.int32)
    tr = Trace()
    rc = lib().lsref_sort_segmented(bits, off, nseg, dt, C.byref(p), C.byref(tr), dec.ctypes.data)
    return out, int(rc), tr, dec[:nseg]


def root_decision(keys: np.ndarray, p: Params | None = None, segment: int = 0):
    """Root-item stage only: (trace, model, splitter, sorted sample)."""
    p = p or params()
    bits, dt = as_bits(keys)
    S = sample_size(bits.size, p)
    s = np.zeros(max(S, 1), dtype=np.uint64)
    tr, m, t = Trace(), Model(), Splitter()
    rc = lib().lsref_root_decision(np.ascontiguousarray(bits), bits.size, dt, C.byref(p), segment,
                                   C.byref(tr), C.byref(m), C.byref(t), s.ctypes.data)
    if rc != OK:
        raise RuntimeError(f"lsref_root_decision failed: {rc}")
    s = s[:S]
    return tr, m, t, (s.view(np.float64) if dt == F64 else s)
