"""Learned SampleSort for GB300 (arxiv 2307.08637): CUDA kernels for sm_103a
behind the C ABI of include/ls.h, with a thin ctypes binding (``ls``).

    import torch, paper_2307_08637_gb300 as lsg
    ctx = lsg.Context(0)
    keys = torch.randn(10**8, dtype=torch.float64, device="cuda")
    stats = lsg.ls_sort(ctx, keys)          # in place, ascending

Importing the package loads liblearnedsort.so and fails loudly if it has not
been built: there is no CPU or library fallback.
"""
from .ls import (  # noqa: F401
    EXPORTS, LIB_PATH, Context, LevelStats, LSError, Model, Params, Stats, lib, ls_classify, ls_classify_static, ls_fit, ls_fit_grad,
    ls_last_device_status, ls_model_export, ls_model_import, ls_params_default, ls_sort, ls_sort_host,
    ls_sort_host_batch, ls_sort_pairs, ls_argsort,
    ls_sort_segmented, ls_workspace_size, status_string, ls_sample, ls_autotune, ls_autotune_segmented, ls_tune_export, ls_tune_import, TuneReport,
    save_tuning, load_tuning, tune_text_to_json, tune_json_to_text,
    LS_OK, LS_EINVAL, LS_ENOMEM, LS_ENAN, LS_ETIMEOUT, LS_ECUDA, LS_ENOTIMPL, LS_EDEVICE,
    LS_F64, LS_U64, LS_PART_AUTO, LS_PART_LEARNED, LS_PART_SPLITTER, LS_RECURSE_REFINE_GLOBAL,
    LS_RECURSE_RETRAIN, LS_CLASSIFY_AUTO, LS_CLASSIFY_DIRECTORY, LS_CLASSIFY_TREE, LS_CLASSIFY_DIRECT, LS_CLASSIFY_GUESS,
    LS_FLAG_DEVICE_LEVELS, LS_FLAG_TIME_PASSES, LS_FLAG_TUNED, LS_LOOP_HOST, LS_LOOP_DEVICE, LS_LOOP_GRAPH,
    LS_LOOP_GRAPH_PDL, PASS_NAMES, PassTime,
    LS_DEC_NONE, LS_DEC_LEARNED, LS_DEC_SPLITTER, LS_DEC_SPLITTER_EQ, LS_DEC_HOMOGENEOUS, LS_DEC_RADIX, LS_MAX_FANOUT,
)

lib()
