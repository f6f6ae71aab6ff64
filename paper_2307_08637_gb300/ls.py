"""ctypes binding of liblearnedsort.so (the C ABI declared in include/ls.h).

Argument marshalling only: every step of a sort runs in the CUDA library.
Functions carry the C names (ls_sort, ls_fit, ...); they take torch CUDA
tensors for device buffers and numpy arrays for host buffers.  Importing
this module loads the shared library and raises if it is missing, so a
product call can never fall back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblearnedsort.so")

LS_OK, LS_EINVAL, LS_ENOMEM, LS_ENAN, LS_ETIMEOUT, LS_ECUDA, LS_ENOTIMPL, LS_EDEVICE = range(8)
LS_F64, LS_U64 = 0, 1
LS_PART_AUTO, LS_PART_LEARNED, LS_PART_SPLITTER = 0, 1, 2
LS_RECURSE_REFINE_GLOBAL, LS_RECURSE_RETRAIN = 0, 1
LS_CLASSIFY_AUTO, LS_CLASSIFY_DIRECTORY, LS_CLASSIFY_TREE, LS_CLASSIFY_DIRECT, LS_CLASSIFY_GUESS = 0, 1, 2, 3, 4
LS_DEC_NONE, LS_DEC_LEARNED, LS_DEC_SPLITTER, LS_DEC_SPLITTER_EQ, LS_DEC_HOMOGENEOUS, LS_DEC_RADIX = 0, 1, 2, 3, 4, 5
LS_MAX_FANOUT = 4096
LS_MAX_LEVELS = 48

# Every function include/ls.h declares.
EXPORTS = (
    "ls_params_default", "ls_create", "ls_destroy", "ls_workspace_size", "ls_sort", "ls_sort_segmented",
    "ls_sort_host", "ls_fit", "ls_classify", "ls_fit_grad", "ls_last_device_status", "ls_model_export",
    "ls_model_import", "ls_status_string", "ls_classify_static", "ls_autotune", "ls_autotune_segmented",
    "ls_tune_export", "ls_tune_import",
    "ls_sort_host_batch", "ls_sort_pairs", "ls_workspace_size_pairs", "ls_last_error_detail", "ls_sample",
)


class LSError(RuntimeError):
    def __init__(self, status: int, what: str):
        detail = lib().ls_last_error_detail().decode() if status in (LS_ECUDA, LS_ENOMEM) else ""
        super().__init__(f"{what} failed: {status_string(status)} ({status})" + (f": {detail}" if detail else ""))
        self.status = status


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
        ("classify_mode", C.c_int32),
        ("tile_keys", C.c_uint32),
        ("flags", C.c_uint32),
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
        ("leaf_x0", C.c_double * LS_MAX_FANOUT),
        ("leaf_a", C.c_double * LS_MAX_FANOUT),
        ("leaf_b", C.c_double * LS_MAX_FANOUT),
        ("leaf_lo", C.c_double * LS_MAX_FANOUT),
        ("leaf_hi", C.c_double * LS_MAX_FANOUT),
        ("leaf_count", C.c_uint32 * LS_MAX_FANOUT),
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


_LEVEL_FIELDS = ("items", "learned", "splitter", "splitter_eq", "homogeneous", "noprogress", "base_items",
                 "base_keys", "fallback_items", "fallback_keys", "keys", "max_child", "sumsq_child", "eq_keys",
                 "radix")


class LevelStats(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in _LEVEL_FIELDS]


LS_FLAG_TIME_PASSES = 1
LS_FLAG_TUNED = 2
LS_FLAG_DEVICE_LEVELS = 4
LS_LOOP_HOST, LS_LOOP_DEVICE, LS_LOOP_GRAPH, LS_LOOP_GRAPH_PDL = 0, 1, 2, 3
PASS_NAMES = ("sample", "fit", "pivots", "classify", "children", "scatter", "base", "copy")


class PassTime(C.Structure):
    _fields_ = [("ms", C.c_double), ("launches", C.c_uint64), ("keys", C.c_uint64)]


class TuneReport(C.Structure):
    _fields_ = [("configs", C.c_uint32), ("base_ms", C.c_double), ("best_ms", C.c_double)]


class Stats(C.Structure):
    _fields_ = [
        ("status", C.c_int32),
        ("root_decision", C.c_int32),
        ("root_sample_size", C.c_uint64),
        ("root_dups", C.c_uint64),
        ("root_imbalance_max", C.c_uint64),
        ("root_nbuckets", C.c_uint32),
        ("levels_used", C.c_uint32),
        ("level", LevelStats * LS_MAX_LEVELS),
        ("ms_total", C.c_double),
        ("kernel_launches", C.c_uint64),
        ("pass_", PassTime * len(PASS_NAMES)),
        ("device_batches", C.c_uint64),
        ("level_loop", C.c_int32),
        ("reserved", C.c_int32),
    ]

    def passes(self) -> dict:
        return {n: {"ms": self.pass_[i].ms, "launches": int(self.pass_[i].launches), "keys": int(self.pass_[i].keys)}
                for i, n in enumerate(PASS_NAMES)}

    def levels(self) -> list[dict]:
        return [{n: int(getattr(self.level[i], n)) for n in _LEVEL_FIELDS} for i in range(self.levels_used)]


_lib = None


def lib() -> C.CDLL:
    """Load liblearnedsort.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
                          " (nvcc, sm_103a); there is no fallback implementation")
    L = C.CDLL(LIB_PATH)
    vp, u64, u32, i32 = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int32
    L.ls_params_default.argtypes = [C.POINTER(Params)]
    L.ls_params_default.restype = None
    L.ls_create.argtypes = [C.POINTER(vp), C.c_int]
    L.ls_create.restype = C.c_int
    L.ls_destroy.argtypes = [vp]
    L.ls_destroy.restype = None
    L.ls_workspace_size.argtypes = [vp, u64, u32, C.c_int, C.POINTER(Params), C.POINTER(C.c_size_t)]
    L.ls_workspace_size.restype = C.c_int
    L.ls_sort.argtypes = [vp, vp, u64, C.c_int, C.POINTER(Params), vp, C.c_size_t, C.POINTER(Stats), vp]
    L.ls_sort.restype = C.c_int
    L.ls_sort_segmented.argtypes = [vp, vp, vp, u32, C.c_int, C.POINTER(Params), vp, C.c_size_t, C.POINTER(Stats),
                                    vp, vp]
    L.ls_sort_segmented.restype = C.c_int
    L.ls_sort_host.argtypes = [vp, vp, u64, C.c_int, C.POINTER(Params), C.POINTER(Stats)]
    L.ls_sort_host.restype = C.c_int
    L.ls_sort_pairs.argtypes = [vp, vp, vp, u32, u64, C.c_int, C.POINTER(Params), vp, C.c_size_t, C.POINTER(Stats),
                                vp]
    L.ls_sort_pairs.restype = C.c_int
    L.ls_workspace_size_pairs.argtypes = [vp, u64, u32, C.c_int, C.POINTER(Params), C.POINTER(C.c_size_t)]
    L.ls_workspace_size_pairs.restype = C.c_int
    L.ls_sort_host_batch.argtypes = [vp, C.POINTER(vp), C.POINTER(u64), u32, C.c_int, C.POINTER(Params),
                                     C.POINTER(Stats)]
    L.ls_sort_host_batch.restype = C.c_int
    L.ls_fit.argtypes = [vp, vp, u64, C.c_int, C.POINTER(Params), C.POINTER(Model), C.POINTER(Stats), vp, vp]
    L.ls_fit.restype = C.c_int
    L.ls_classify.argtypes = [vp, C.POINTER(Model), vp, u64, C.c_int, u32, u64, i32, vp, vp, vp]
    L.ls_classify.restype = C.c_int
    L.ls_classify_static.argtypes = [C.POINTER(Model), vp, u64, C.c_int, u32, u64, i32, vp, vp, vp]
    L.ls_classify_static.restype = C.c_int
    L.ls_fit_grad.argtypes = [vp, C.POINTER(Model), vp, u64, C.c_int, vp, vp, vp, vp, vp, vp]
    L.ls_fit_grad.restype = C.c_int
    L.ls_last_device_status.argtypes = [vp, vp]
    L.ls_last_device_status.restype = C.c_int
    L.ls_model_export.argtypes = [C.POINTER(Model), vp, C.POINTER(C.c_size_t)]
    L.ls_model_export.restype = C.c_int
    L.ls_model_import.argtypes = [C.POINTER(Model), vp, C.c_size_t]
    L.ls_model_import.restype = C.c_int
    L.ls_status_string.argtypes = [C.c_int]
    L.ls_status_string.restype = C.c_char_p
    L.ls_last_error_detail.argtypes = []
    L.ls_last_error_detail.restype = C.c_char_p
    L.ls_sample.argtypes = [vp, vp, u64, C.c_int, u64, u64, vp, vp]
    L.ls_sample.restype = C.c_int
    L.ls_autotune.argtypes = [vp, vp, u64, C.c_int, C.POINTER(Params), C.POINTER(Params), C.POINTER(TuneReport), vp]
    L.ls_autotune.restype = C.c_int
    L.ls_autotune_segmented.argtypes = [vp, vp, C.POINTER(C.c_uint64), C.c_uint32, C.c_int, C.POINTER(Params),
                                        C.POINTER(Params), C.POINTER(TuneReport), vp]
    L.ls_autotune_segmented.restype = C.c_int
    L.ls_tune_export.argtypes = [vp, C.c_char_p, C.POINTER(C.c_size_t)]
    L.ls_tune_export.restype = C.c_int
    L.ls_tune_import.argtypes = [vp, C.c_char_p]
    L.ls_tune_import.restype = C.c_int
    _lib = L
    return L


def status_string(s: int) -> str:
    return lib().ls_status_string(int(s)).decode()


def _check(rc: int, what: str) -> None:
    if rc != LS_OK:
        raise LSError(rc, what)


def ls_params_default(**overrides) -> Params:
    p = Params()
    lib().ls_params_default(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


# ------------------------------------------------------------ tensor helpers

def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return LS_F64
    if t.dtype in (torch.uint64, torch.int64):
        return LS_U64
    raise TypeError(f"keys must be float64 or uint64, got {t.dtype}")


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Context:
    """An ls_ctx bound to one CUDA device (ls_create / ls_destroy)."""

    def __init__(self, device: int = 0):
        self.device = device
        self._h = C.c_void_p()
        _check(lib().ls_create(C.byref(self._h), device), "ls_create")
        self._ws = None

    def close(self):
        if self._h:
            lib().ls_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def free_workspace(self):
        """Drop the cached workspace tensor (its memory returns to torch's allocator)."""
        self._ws = None

    def workspace_bytes(self, nbytes: int):
        """A cached device workspace of at least nbytes."""
        import torch
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = None
            self._ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=f"cuda:{self.device}")
        return self._ws

    def workspace(self, n: int, nseg: int, dtype: int, p: Params):
        import torch
        nbytes = ls_workspace_size(self, n, nseg, dtype, p)
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = None
            self._ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=f"cuda:{self.device}")
        return self._ws


def ls_workspace_size(ctx: Context, n: int, nseg: int, dtype: int, p: Params) -> int:
    out = C.c_size_t()
    _check(lib().ls_workspace_size(ctx.handle if ctx else None, n, nseg, dtype, C.byref(p), C.byref(out)),
           "ls_workspace_size")
    return out.value


def ls_sort(ctx: Context, keys, p: Params | None = None, workspace=None, stream=None, check: bool = True) -> Stats:
    """Sort a CUDA float64/uint64 tensor in place; returns the call's statistics."""
    p = p or ls_params_default()
    dt = _dtype_code(keys)
    n = keys.numel()
    ws = workspace if workspace is not None else ctx.workspace(n, 1, dt, p)
    st = Stats()
    rc = lib().ls_sort(ctx.handle, _ptr(keys), n, dt, C.byref(p), _ptr(ws), ws.numel(), C.byref(st), _stream(stream))
    if check:
        _check(rc, "ls_sort")
    st.status = rc if rc else st.status
    return st


def ls_sort_pairs(ctx: Context, keys, vals, p: Params | None = None, stream=None, check: bool = True) -> Stats:
    """Sort keys in place and permute vals (4- or 8-byte elements, same length)
    the same way; stable for equal keys."""
    p = p or ls_params_default()
    dt = _dtype_code(keys)
    n = keys.numel()
    if vals.numel() != n or vals.element_size() not in (4, 8) or not vals.is_contiguous():
        raise ValueError("vals must be a contiguous tensor of n 4- or 8-byte elements")
    vb = vals.element_size()
    nb = C.c_size_t()
    _check(lib().ls_workspace_size_pairs(ctx.handle, n, vb, dt, C.byref(p), C.byref(nb)), "ls_workspace_size_pairs")
    ws = ctx.workspace_bytes(nb.value)
    st = Stats()
    rc = lib().ls_sort_pairs(ctx.handle, _ptr(keys), _ptr(vals), vb, n, dt, C.byref(p), _ptr(ws), ws.numel(),
                             C.byref(st), _stream(stream))
    if check:
        _check(rc, "ls_sort_pairs")
    return st


def ls_argsort(ctx: Context, keys, p: Params | None = None, stream=None):
    """Sort keys in place and return the stable argsort of the original keys
    (int64 indices: sorted[i] = original[idx[i]])."""
    import torch
    n = keys.numel()
    idx = torch.arange(n, dtype=torch.int32 if n < 2**31 else torch.int64, device=keys.device)
    ls_sort_pairs(ctx, keys, idx, p, stream)
    return idx.long()


def ls_sort_segmented(ctx: Context, keys, offsets, p: Params | None = None, workspace=None, stream=None,
                      check: bool = True):
    """Sort each keys[off[s]:off[s+1]] independently; returns (stats, per-segment decisions)."""
    p = p or ls_params_default()
    dt = _dtype_code(keys)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
    nseg = off.size - 1
    ws = workspace if workspace is not None else ctx.workspace(keys.numel(), nseg, dt, p)
    dec = np.zeros(max(nseg, 1), dtype=np.int32)
    st = Stats()
    rc = lib().ls_sort_segmented(ctx.handle, _ptr(keys), off.ctypes.data, nseg, dt, C.byref(p), _ptr(ws), ws.numel(),
                                 C.byref(st), dec.ctypes.data, _stream(stream))
    if check:
        _check(rc, "ls_sort_segmented")
    return st, dec[:nseg]


def ls_sort_host(ctx: Context, keys: np.ndarray, p: Params | None = None) -> Stats:
    """End-to-end sort of a host numpy array (float64 or uint64), in place."""
    p = p or ls_params_default()
    if keys.dtype == np.float64:
        dt = LS_F64
    elif keys.dtype == np.uint64:
        dt = LS_U64
    else:
        raise TypeError(keys.dtype)
    if not keys.flags["C_CONTIGUOUS"]:
        raise ValueError("keys must be contiguous")
    st = Stats()
    _check(lib().ls_sort_host(ctx.handle, keys.ctypes.data, keys.size, dt, C.byref(p), C.byref(st)), "ls_sort_host")
    return st


def ls_sort_host_batch(ctx: Context, arrays, p: Params | None = None, stats: bool = False):
    """Sort several host numpy arrays (float64 or uint64, one dtype) in place,
    copies pipelined with the sorts; returns the per-array Stats when asked."""
    p = p or ls_params_default()
    arrays = list(arrays)
    if not arrays:
        return [] if stats else None
    kinds = {a.dtype for a in arrays}
    if len(kinds) != 1 or arrays[0].dtype not in (np.float64, np.uint64):
        raise TypeError("arrays must all be float64 or all uint64")
    for a in arrays:
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
    dt = LS_F64 if arrays[0].dtype == np.float64 else LS_U64
    cnt = len(arrays)
    ptrs = (C.c_void_p * cnt)(*[a.ctypes.data for a in arrays])
    ns = (C.c_uint64 * cnt)(*[a.size for a in arrays])
    st = (Stats * cnt)() if stats else None
    _check(lib().ls_sort_host_batch(ctx.handle, ptrs, ns, cnt, dt, C.byref(p), st), "ls_sort_host_batch")
    return list(st) if stats else None


def ls_fit(ctx: Context, keys, p: Params | None = None, want_sample: bool = False, stream=None):
    """Train the root RMI as ls_sort would; returns (Model, Stats, sorted sample tensor|None)."""
    import torch
    p = p or ls_params_default()
    dt = _dtype_code(keys)
    m = Model()
    st = Stats()
    samp = None
    if want_sample:
        n = keys.numel()
        import math
        S = n if not (math.ceil(p.sample_rate * n) < n) else max(int(math.ceil(p.sample_rate * n)), 0)
        S = min(n, max(S, p.min_sample))
        samp = torch.empty(S, dtype=keys.dtype, device=keys.device)
    _check(lib().ls_fit(ctx.handle, _ptr(keys), keys.numel(), dt, C.byref(p), C.byref(m), C.byref(st), _ptr(samp),
                        _stream(stream)), "ls_fit")
    return m, st, samp


def ls_classify(ctx: Context, model: Model, keys, k: int = 0, g: int = 0, mode: int = LS_CLASSIFY_AUTO,
                want_ids: bool = True, stream=None):
    """Bucket ids (uint32 as int32 tensor) and histogram (int64 tensor) of keys under `model`."""
    import torch
    dt = _dtype_code(keys)
    ids = torch.empty(keys.numel(), dtype=torch.int32, device=keys.device) if want_ids else None
    hist = torch.zeros(model.L, dtype=torch.int64, device=keys.device)
    _check(lib().ls_classify(ctx.handle, C.byref(model), _ptr(keys), keys.numel(), dt, k, g, mode, _ptr(ids),
                             _ptr(hist), _stream(stream)), "ls_classify")
    return ids, hist


def ls_classify_static(model: Model, keys, ids, hist, k: int = 0, g: int = 0, mode: int = LS_CLASSIFY_AUTO,
                       stream=None) -> None:
    """ls_classify into caller-provided outputs, with no device allocation
    anywhere on the path (for callers that cannot allocate: see ls.h).

    The C entry point trusts its pointers, so the tensors are checked here:
    keys float64 / uint64 (int64 bit patterns accepted), ids int32 with at
    least keys.numel() elements (or None), hist int64 with at least model.L
    elements (or None), all contiguous CUDA tensors on keys' device.  The
    call runs with that device current, on `stream` or that device's current
    stream."""
    import torch
    if not isinstance(keys, torch.Tensor) or not keys.is_cuda:
        raise ValueError("keys must be a CUDA tensor")
    dt = _dtype_code(keys)
    if not keys.is_contiguous():
        raise ValueError("keys must be contiguous")
    dev = keys.device
    for name, t, dtype, need in (("ids", ids, torch.int32, keys.numel()), ("hist", hist, torch.int64, model.L)):
        if t is None:
            continue
        if not isinstance(t, torch.Tensor) or t.device != dev:
            raise ValueError(f"{name} must be a CUDA tensor on {dev}")
        if t.dtype != dtype:
            raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() < need:
            raise ValueError(f"{name} holds {t.numel()} elements, needs {need}")
    with torch.cuda.device(dev):
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        _check(lib().ls_classify_static(C.byref(model), _ptr(keys), keys.numel(), dt, k, g, mode, _ptr(ids),
                                        _ptr(hist), _stream(st)), "ls_classify_static")


def ls_sample(ctx: Context, keys, S: int, seed: int, stream=None):
    """Sample(A): min(S, n) keys of `keys` drawn with replacement from the
    counter-based SplitMix64 stream at `seed` (a new tensor, same dtype)."""
    import torch
    dt = _dtype_code(keys)
    if not keys.is_contiguous():
        raise ValueError("keys must be contiguous")
    n = keys.numel()
    out = torch.empty(min(S, n), dtype=keys.dtype, device=keys.device)
    _check(lib().ls_sample(ctx.handle, _ptr(keys), n, dt, S, seed % 2**64, _ptr(out), _stream(stream)), "ls_sample")
    return out


def ls_fit_grad(ctx: Context, model: Model, sorted_sample, stream=None) -> dict:
    """Forward (pred, resid) and backward (grad_a, grad_b, grad_root) of the fit objective."""
    import torch
    dt = _dtype_code(sorted_sample)
    S = sorted_sample.numel()
    dev = sorted_sample.device
    out = {
        "pred": torch.empty(S, dtype=torch.float64, device=dev),
        "resid": torch.empty(S, dtype=torch.float64, device=dev),
        "grad_a": torch.empty(model.L, dtype=torch.float64, device=dev),
        "grad_b": torch.empty(model.L, dtype=torch.float64, device=dev),
        "grad_root": torch.empty(2, dtype=torch.float64, device=dev),
    }
    _check(lib().ls_fit_grad(ctx.handle, C.byref(model), _ptr(sorted_sample), S, dt, _ptr(out["pred"]),
                             _ptr(out["resid"]), _ptr(out["grad_a"]), _ptr(out["grad_b"]), _ptr(out["grad_root"]),
                             _stream(stream)), "ls_fit_grad")
    return out


def ls_last_device_status(ctx: Context, stream=None) -> int:
    return int(lib().ls_last_device_status(ctx.handle, _stream(stream)))


def ls_model_export(m: Model) -> bytes:
    n = C.c_size_t()
    _check(lib().ls_model_export(C.byref(m), None, C.byref(n)), "ls_model_export")
    buf = C.create_string_buffer(n.value)
    _check(lib().ls_model_export(C.byref(m), buf, C.byref(n)), "ls_model_export")
    return buf.raw[: n.value]


def ls_model_import(data: bytes) -> Model:
    m = Model()
    buf = C.create_string_buffer(data, len(data))
    _check(lib().ls_model_import(C.byref(m), buf, len(data)), "ls_model_import")
    return m


def ls_autotune(ctx: Context, keys, base: Params | None = None, stream=None) -> tuple[Params, TuneReport]:
    """Time candidate (fanout, base-case threshold, sample rate, recursion)
    settings on copies of `keys` (not modified) and return the fastest, which
    is also stored in the context for LS_FLAG_TUNED."""
    base = base or ls_params_default()
    out = Params()
    rep = TuneReport()
    rc = lib().ls_autotune(ctx.handle, _ptr(keys), keys.numel(), _dtype_code(keys), C.byref(base), C.byref(out),
                           C.byref(rep), _stream(stream))
    _check(rc, "ls_autotune")
    return out, rep


def ls_autotune_segmented(ctx: Context, keys, offsets, base: Params | None = None,
                          stream=None) -> tuple[Params, TuneReport]:
    """ls_autotune for the segmented form: candidates are timed on
    ls_sort_segmented of copies of keys[:offsets[-1]] split at `offsets`
    (offsets[0] = 0); the winner is stored for the mean segment length."""
    base = base or ls_params_default()
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
    if off.ndim != 1 or off.size < 2 or int(off[-1]) > keys.numel():
        raise ValueError("offsets must be nseg + 1 non-decreasing values within the keys")
    out = Params()
    rep = TuneReport()
    rc = lib().ls_autotune_segmented(ctx.handle, _ptr(keys), off.ctypes.data_as(C.POINTER(C.c_uint64)), off.size - 1,
                                     _dtype_code(keys), C.byref(base), C.byref(out), C.byref(rep), _stream(stream))
    _check(rc, "ls_autotune_segmented")
    return out, rep


def ls_tune_export(ctx: Context) -> str:
    """The context's tuning table as text (one entry per line)."""
    n = C.c_size_t(0)
    _check(lib().ls_tune_export(ctx.handle, None, C.byref(n)), "ls_tune_export")
    buf = C.create_string_buffer(n.value)
    _check(lib().ls_tune_export(ctx.handle, buf, C.byref(n)), "ls_tune_export")
    return buf.value.decode()


def ls_tune_import(ctx: Context, text: str) -> None:
    """Add / replace tuning entries from ls_tune_export text."""
    _check(lib().ls_tune_import(ctx.handle, text.encode()), "ls_tune_import")


_TUNE_FIELDS = ("dtype", "log2n", "fanout", "basecase_threshold", "sample_rate", "recurse_model", "ms")


def tune_text_to_json(text: str) -> list[dict]:
    """Parse ls_tune_export text into JSON-ready records."""
    out = []
    for line in text.splitlines():
        if not line.strip():
            continue
        v = line.split()
        if len(v) != len(_TUNE_FIELDS):
            raise ValueError(f"bad tuning line: {line!r}")
        out.append({"dtype": int(v[0]), "log2n": int(v[1]), "fanout": int(v[2]), "basecase_threshold": int(v[3]),
                    "sample_rate": float(v[4]), "recurse_model": int(v[5]), "ms": float(v[6])})
    return out


def tune_json_to_text(records: list[dict]) -> str:
    """Inverse of tune_text_to_json (the text ls_tune_import reads)."""
    return "".join(f"{int(r['dtype'])} {int(r['log2n'])} {int(r['fanout'])} {int(r['basecase_threshold'])} "
                   f"{float(r['sample_rate']):.17g} {int(r['recurse_model'])} {float(r['ms']):.6f}\n" for r in records)


def save_tuning(ctx: Context, path: str) -> None:
    """Write the context's tuning table to a JSON file."""
    import json
    with open(path, "w") as f:
        json.dump(tune_text_to_json(ls_tune_export(ctx)), f, indent=1)


def load_tuning(ctx: Context, path: str) -> None:
    """Load a JSON tuning table written by save_tuning into the context."""
    import json
    with open(path) as f:
        ls_tune_import(ctx, tune_json_to_text(json.load(f)))
