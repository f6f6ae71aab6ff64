"""Benchmark: full sorts of 1e8 float64 keys on one GB300, learned vs splitter.

A step sorts six 1e8-key float64 arrays, one per synthetic distribution of
the paper's suite (normal, lognormal, exponential, chi-squared, mixture of 5
Gaussians, uniform on [0, 1e6)), each through ls_sort on the device, with the
partitioner Alg. 5 picks (the RMI for all six).  The same arrays are then
sorted with the splitter tree forced, on the same kernels.  Every sort
starts from the unsorted input: a device-to-device restore copy runs before
each sort, outside its CUDA-event pair.  The inputs (800 MB each) are larger
than L2 (129 MB), so no flush is needed.

Printed on rank 0: one JSON line (metric keys/s).  `--impl reference` times
the CPU oracle instead (single thread, bounded samples).  Under torchrun every
rank sorts its own six arrays (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import datagen  # noqa: E402

METRIC = "keys/s and % HBM roofline at 1e8 f64 keys, learned vs splitter partition, 1 GB300"
DISTS = datagen.F64_DISTS
FALLBACK_HBM_GBS = 6800.0
SCATTER_BYTES_PER_KEY = 16  # K3 reads each key once and writes it once
CLASSIFY_BYTES_PER_KEY = 8  # K1 reads each key once
BASECASE_T = 4096           # buckets of <= 4096 keys go to the shared-memory base case
TUNE_SEGS = 512             # C4: segments the autotuner times the segmented sort on


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=float, default=1e8)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-splitter", action="store_true")
    ap.add_argument("--no-device-levels", action="store_true",
                    help="leave out the C2 sorts with the levels below the root planned on the device")
    ap.add_argument("--dists", default=",".join(DISTS), help="comma-separated subset (profiling runs)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c4"],
                    help="c2: six 1e8-key arrays (the headline); c4: 4096 segments, batched vs one call per array")
    ap.add_argument("--nseg", type=int, default=4096, help="c4: number of segments")
    ap.add_argument("--no-c4", action="store_true", help="leave the C4 batch out of the default line")
    ap.add_argument("--no-c5", action="store_true", help="leave the C5 2e9-key run out of the default line")
    ap.add_argument("--c5-n", type=float, default=2e9, help="C5 keys")
    ap.add_argument("--classify", default="auto", choices=["auto", "guess", "directory", "tree"],
                    help="pivot-table evaluation mode of the learned classifier (ls_classify_mode)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(seed, rank):
    """Seed of one rank's arrays: every rank sorts its own inputs (weak scaling)."""
    return seed + 1000 * rank


def max_over_ranks(x, world, device):
    """The slowest rank's value, agreed by all ranks (all-reduce MAX); x on one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_keys_per_s(world, keys_per_step, step_ms):
    """Whole-job throughput: every rank's keys over the slowest rank's step time."""
    return world * keys_per_step / (step_ms / 1e3)


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def k3b_source_sha256(text: str) -> str:
    """sha256 of the buffered scatter kernel's section of ls_partition.cu
    (from its constants up to the chunk-prefix section)."""
    a = text.index("constexpr uint32_t kBufTPB")
    b = text.index("// ------------------------------------------------------------------ chunk prefixes", a)
    return hashlib.sha256(text[a:b].encode()).hexdigest()


def ncu_traffic():
    """DRAM bytes per key of the buffered scatter kernel (K3b) from the
    committed ncu summary, only while the kernel's source is unchanged since
    the capture."""
    path = os.path.join(ROOT, "profiles", "scatter_traffic.json")
    src = os.path.join(ROOT, "paper_2307_08637_gb300", "csrc", "ls_partition.cu")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("kernel_source_sha256") != k3b_source_sha256(open(src).read()):
            return None
        return float(d["dram_bytes_per_key"])
    except Exception:
        return None


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, dev: int):
        self.dev = dev
        self.proc = None
        # the raw samples: LS_CLOCKS_DIR if set (to keep them), else a temporary directory
        out_dir = os.environ.get("LS_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_gpu{dev}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        try:
            rows = [l.strip().split(", ") for l in open(self.path) if l.strip()]
        except Exception:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def gen_inputs(n: int, seed: int, dists=DISTS):
    return [(d, datagen.generate(d, n, seed)) for d in dists]


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    n = int(args.n)
    # a step is one whole array of the C2 workload (the six distributions in
    # turn), sorted with the same parameters as the GPU arm; ~5 s per 1e8 keys
    # on one core, so the default 3 + 5 steps take well under a minute per step
    inputs = gen_inputs(n, args.seed)
    p = oracle.params(basecase_threshold=BASECASE_T)
    times = []
    for step in range(args.warmup + args.steps):
        d, x = inputs[step % len(inputs)]
        t0 = time.perf_counter()
        out, rc, tr, _, _ = oracle.sort(x, p)
        dt = time.perf_counter() - t0
        assert rc == 0
        if step >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = n * len(times) / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "C2: one whole 1e8-key float64 array per step, the six distributions in turn, "
                               "same parameters as the GPU arm (fanout 1000, sample 1 %, T = 4096, REFINE_GLOBAL)",
                   "distributions": list(DISTS), "keys_per_step": n},
        "cpu_baseline": {"value": value, "unit": "keys/s", "cores": 1, "kind": "oracle",
                         "sample": f"{n} keys per step (one whole array), distributions cycled"},
        "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def time_sorts(lsg, ctx, work, pristine, p, torch, stream):
    """Sort every array once from its pristine copy; returns (ms list, stats list)."""
    ms, sts = [], []
    for w, src in zip(work, pristine):
        w.copy_(src)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = lsg.ls_sort(ctx, w, p, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        sts.append(st)
    return ms, sts


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)
    import paper_2307_08637_gb300 as lsg

    n = int(args.n)
    stream = torch.cuda.current_stream()
    ctx = lsg.Context(dev)
    dists = tuple(d for d in args.dists.split(",") if d)
    inputs = gen_inputs(n, rank_seed(args.seed, rank), dists)
    pristine = [torch.from_numpy(x).to(f"cuda:{dev}") for _, x in inputs]
    work = [torch.empty_like(t) for t in pristine]
    cmode = {"auto": lsg.LS_CLASSIFY_AUTO, "guess": lsg.LS_CLASSIFY_GUESS, "directory": lsg.LS_CLASSIFY_DIRECTORY,
             "tree": lsg.LS_CLASSIFY_TREE}[args.classify]
    # the timed sorts run untimed inside (levels below the root as one CUDA
    # graph); the per-pass breakdown comes from separate instrumented sorts
    # (LS_FLAG_TIME_PASSES: the same kernels, launched batch by batch from
    # the host so that CUDA events can bracket each pass)
    p_learned = lsg.ls_params_default(basecase_threshold=BASECASE_T, classify_mode=cmode)
    p_learned_t = lsg.ls_params_default(flags=lsg.LS_FLAG_TIME_PASSES, basecase_threshold=BASECASE_T,
                                        classify_mode=cmode)
    p_split = lsg.ls_params_default(flags=lsg.LS_FLAG_TIME_PASSES, partitioner=lsg.LS_PART_SPLITTER,
                                    basecase_threshold=BASECASE_T, classify_mode=cmode)
    ctx.workspace(n, 1, lsg.LS_F64, p_split)  # allocate once, before timing

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        time_sorts(lsg, ctx, work, pristine, p_learned, torch, stream)
    barrier()
    ms_learned, sts_learned = [], []
    with Clocks(dev) as clk:
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            ms, sts = time_sorts(lsg, ctx, work, pristine, p_learned, torch, stream)
            ms_learned.append(sum(ms))
            sts_learned += sts
        barrier()
        wall = time.perf_counter() - wall0
    # correctness guard on the last sorted array of the timed region
    last = work[-1]
    sord = last.view(torch.int64)
    sord = sord ^ ((sord >> 63) & 0x7FFFFFFFFFFFFFFF)
    assert bool((sord[1:] >= sord[:-1]).all()), "bench output not sorted"
    step_ms = max_over_ranks(sum(ms_learned) / len(ms_learned), world, f"cuda:{dev}")
    keys_per_step = n * len(inputs)
    value = job_keys_per_s(world, keys_per_step, step_ms)

    # per-pass device time: instrumented sorts of the same arrays
    prof_steps = max(1, min(args.steps, 3))
    sts_prof = []
    for _ in range(prof_steps):
        sts_prof += time_sorts(lsg, ctx, work, pristine, p_learned_t, torch, stream)[1]
    passes = {}
    for st in sts_prof:
        for k, v in st.passes().items():
            a = passes.setdefault(k, {"ms": 0.0, "launches": 0, "keys": 0})
            a["ms"] += v["ms"]
            a["launches"] += v["launches"]
            a["keys"] += v["keys"]
    peak, peak_kind = measured_peak()
    sc = passes["scatter"]
    achieved = SCATTER_BYTES_PER_KEY * sc["keys"] / (sc["ms"] / 1e3) / 1e9 if sc["ms"] > 0 else None
    k1 = passes["classify"]
    k1_gbs = CLASSIFY_BYTES_PER_KEY * k1["keys"] / (k1["ms"] / 1e3) / 1e9 if k1["ms"] > 0 else None
    tr = ncu_traffic()
    roofline = {
        "kernel": "k_scatter_buffered (K3b buffered partition scatter: every C2 item is learned under "
                  "REFINE_GLOBAL or a radix split, so the scatter pass is K3b)",
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": achieved / peak if achieved else None, "peak_source": peak_kind,
        "bytes_per_key": SCATTER_BYTES_PER_KEY,
        "keys_per_launch": sc["keys"] / max(sc["launches"], 1),
        "traffic": (tr * sc["keys"] / max(sc["launches"], 1)) if tr else None,
        "frac_of_8TBps": achieved / 8000.0 if achieved else None,
        "classify_k1_gbs": k1_gbs, "classify_k1_frac": (k1_gbs / peak) if k1_gbs else None,
    }
    # per-distribution details of the timed learned sorts
    per_dist = {}
    for i, (d, _) in enumerate(inputs):
        tms = [st.ms_total for st in sts_learned[i::len(inputs)]]
        per_dist[d] = {"host_ms_mean": sum(tms) / len(tms), "root_decision": int(sts_learned[i].root_decision),
                       "levels": int(sts_learned[i].levels_used),
                       "level1_max_bucket": int(sts_learned[i].level[0].max_child),
                       "level1_bucket_sumsq": int(sts_learned[i].level[0].sumsq_child)}

    split = None
    if not args.no_splitter:
        ms_s, sts_s = [], []
        for _ in range(max(1, args.steps // 2)):
            ms, sts = time_sorts(lsg, ctx, work, pristine, p_split, torch, stream)
            ms_s.append(sum(ms))
            sts_s += sts
        s_ms = max_over_ranks(sum(ms_s) / len(ms_s), world, f"cuda:{dev}")
        ps = {}
        for st in sts_s:
            for k, v in st.passes().items():
                a = ps.setdefault(k, {"ms": 0.0, "keys": 0})
                a["ms"] += v["ms"]
                a["keys"] += v["keys"]
        split = {"value": job_keys_per_s(world, keys_per_step, s_ms), "unit": "keys/s", "ms_per_step": s_ms,
                 "learned_speedup": s_ms / step_ms,
                 "scatter_gbs": SCATTER_BYTES_PER_KEY * ps["scatter"]["keys"] / (ps["scatter"]["ms"] / 1e3) / 1e9,
                 "classify_gbs": CLASSIFY_BYTES_PER_KEY * ps["classify"]["keys"] / (ps["classify"]["ms"] / 1e3) / 1e9,
                 "passes_ms_per_step": {k: v["ms"] / len(ms_s) for k, v in ps.items()},
                 "level1_max_bucket": {d: int(sts_s[i].level[0].max_child) for i, (d, _) in enumerate(inputs)},
                 "level1_bucket_sumsq": {d: int(sts_s[i].level[0].sumsq_child) for i, (d, _) in enumerate(inputs)}}

    # the same sorts with the levels below the root planned on the device
    # (device work queue, one CUDA graph per array: captured in the first
    # untimed round, then reused)
    devlv = None
    if not args.no_device_levels:
        p_dev = lsg.ls_params_default(flags=lsg.LS_FLAG_DEVICE_LEVELS, basecase_threshold=BASECASE_T,
                                      classify_mode=cmode)
        time_sorts(lsg, ctx, work, pristine, p_dev, torch, stream)
        ms_d, sts_d = [], []
        for _ in range(max(1, min(args.steps, 3))):
            ms, sts = time_sorts(lsg, ctx, work, pristine, p_dev, torch, stream)
            ms_d.append(sum(ms))
            sts_d += sts
        d_ms = max_over_ranks(sum(ms_d) / len(ms_d), world, f"cuda:{dev}")
        devlv = {"value": job_keys_per_s(world, keys_per_step, d_ms), "unit": "keys/s", "ms_per_step": d_ms,
                 "vs_host_planned": step_ms / d_ms,
                 "level_loop": sorted({int(st.level_loop) for st in sts_d}),
                 "device_batches_per_sort": sum(int(st.device_batches) for st in sts_d) / len(sts_d),
                 "gpu_launches_per_sort": sum(int(st.kernel_launches) for st in sts_d) / len(sts_d)}

    e2e = None
    if not args.no_e2e:
        # the public host API: ls_sort_host_batch over the step's six arrays
        # (copies in and out pipelined against the sorts), from page-locked
        # host buffers restored before each timed step
        host = [torch.from_numpy(x).pin_memory().numpy() for _, x in inputs]
        host_src = [x.copy() for _, x in inputs]
        p_plain = lsg.ls_params_default(basecase_threshold=BASECASE_T)
        lsg.ls_sort_host_batch(ctx, host, p_plain)  # warm the context's device cache and streams
        tt = []
        for _ in range(max(1, min(args.steps, 3))):
            for h, src in zip(host, host_src):
                np.copyto(h, src)
            t0 = time.perf_counter()
            lsg.ls_sort_host_batch(ctx, host, p_plain)
            tt.append(time.perf_counter() - t0)
        for h, src in zip(host, host_src):  # ascending, and the same multiset of bit patterns
            hb, sb = h.view(np.uint64), src.view(np.uint64)
            assert bool(np.all(h[1:] >= h[:-1])), "end-to-end output not sorted"
            assert hb.sum(dtype=np.uint64) == sb.sum(dtype=np.uint64)
            assert np.bitwise_xor.reduce(hb) == np.bitwise_xor.reduce(sb)
        e2e_ms = max_over_ranks(1e3 * sum(tt) / len(tt), world, f"cuda:{dev}")
        e2e = {"value": job_keys_per_s(world, keys_per_step, e2e_ms), "unit": "keys/s",
               "h2d_bytes_per_step": 8 * keys_per_step, "d2h_bytes_per_step": 8 * keys_per_step,
               "ms_per_step": e2e_ms,
               "api": "ls_sort_host_batch (six page-locked host arrays, copies pipelined with the sorts)"}

    cpu = None
    if not args.no_cpu and rank == 0:
        import oracle

        oracle.build()
        # mean of 3 runs on a bounded sample: the first 1e7 keys of three of
        # the six arrays (the oracle is single-threaded; ~5 s per 1e8 keys)
        runs = []
        for d, x in inputs[:3]:
            xs = x[:min(x.size, 10_000_000)]
            t0 = time.perf_counter()
            out, rc, _, _, _ = oracle.sort(xs, oracle.params(basecase_threshold=BASECASE_T))
            runs.append((xs.size, time.perf_counter() - t0))
            assert rc == 0
        cpu = {"value": statistics.mean(k / t for k, t in runs), "unit": "keys/s", "cores": 1, "kind": "oracle",
               "sample": "mean of 3 runs, each the first 1e7 keys of one array (" +
                         ", ".join(d for d, _ in inputs[:3]) + "), single thread",
               "seconds": [t for _, t in runs]}

    launches = sum(int(st.kernel_launches) for st in sts_learned)
    # the other configurations, measured on the same GPU after the headline
    # (single-rank runs only: the scaling runs repeat the headline alone)
    c4 = c5 = None
    if world == 1 and not (args.no_c4 and args.no_c5):
        del pristine, work
        ctx.free_workspace()
        torch.cuda.empty_cache()
        if not args.no_c4:
            c4 = c4_measure(lsg, ctx, args, torch, stream, with_cpu=False)
            ctx.free_workspace()
            torch.cuda.empty_cache()
        if not args.no_c5:
            c5 = c5_measure(lsg, ctx, args, torch, stream)
            ctx.free_workspace()
            torch.cuda.empty_cache()
    line = {
        "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "C2: six 1e8-key float64 arrays per step (normal, lognormal, exponential, "
                               "chi-squared, mix of 5 Gaussians, uniform[0,1e6)), full sort each",
                   "partitioner": "Alg. 5 AUTO (RMI chosen on all six)", "fanout": 1000, "sample_rate": 0.01,
                   "basecase_threshold": BASECASE_T, "recurse": "REFINE_GLOBAL",
                   "keys_per_step_per_gpu": keys_per_step, "l2": "inputs 800 MB each, larger than L2; no flush",
                   "timing": "CUDA events around each ls_sort on the launching stream; D2D input restore outside; "
                             "per-pass times (roofline, passes_ms_per_step) from %d further instrumented steps "
                             "(LS_FLAG_TIME_PASSES)" % prof_steps,
                   "wall_s_timed_region_incl_restores": wall},
        "roofline": roofline,
        "splitter": split,
        "device_levels": devlv,
        "per_dist": per_dist,
        "passes_ms_per_step": {k: v["ms"] / prof_steps for k, v in passes.items()},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk.summary(),
        "gpu_launches": launches,
        "c4": c4,
        "c5": c5,
    }
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _oracle_segments(args_tuple):
    """One oracle sort per segment (worker of the multi-core C4 baseline)."""
    import oracle

    x, kw = args_tuple
    out, rc, _, _, _ = oracle.sort(x, oracle.params(**kw))
    return rc


def c4_measure(lsg, ctx, args, torch, stream, with_cpu=True):
    """C4: nseg float64 arrays with log-uniform lengths in [1e3, 1e6], each its
    own distribution with a random affine map; one ls_sort_segmented call
    (every segment's sample, model and partition handled level by level in
    shared launches) against one ls_sort call per array, both with the
    parameters the autotuner picks on a segment of the mean length."""
    dev = 0
    keys, off, names = datagen.segmented(args.nseg, 4)
    nseg = off.size - 1
    n = int(off[-1])
    pristine = torch.from_numpy(keys).to(f"cuda:{dev}")
    work = torch.empty_like(pristine)
    # parameters tuned on the segmented form itself (the first TUNE_SEGS
    # segments: the lengths are i.i.d., so their mix is the batch's)
    tseg = min(TUNE_SEGS, nseg)
    base = lsg.ls_params_default()
    tuned, rep = lsg.ls_autotune_segmented(ctx, pristine[:int(off[tseg])], off[:tseg + 1], base)
    p = lsg.ls_params_default(fanout=tuned.fanout, basecase_threshold=tuned.basecase_threshold,
                              sample_rate=tuned.sample_rate, recurse_model=tuned.recurse_model)
    ctx.workspace(n, nseg, lsg.LS_F64, p)

    def batched():
        work.copy_(pristine)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, dec = lsg.ls_sort_segmented(ctx, work, off, p, stream=stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), st

    def looped():
        work.copy_(pristine)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        launches = 0
        for s in range(nseg):
            st = lsg.ls_sort(ctx, work[int(off[s]):int(off[s + 1])], p, stream=stream)
            launches += int(st.kernel_launches)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), launches

    for _ in range(max(1, min(args.warmup, 3))):
        batched()
    torch.cuda.synchronize()
    with Clocks(dev) as clk:
        bms, bst = [], None
        for _ in range(max(1, min(args.steps, 5))):
            ms, bst = batched()
            bms.append(ms)
    out_b = work.clone()
    # every segment ascending under ord
    o = out_b.view(torch.int64)
    o = o ^ ((o >> 63) & 0x7FFFFFFFFFFFFFFF)
    ok = (o[1:] >= o[:-1])
    starts = torch.from_numpy(off[1:-1].astype(np.int64) - 1).to(f"cuda:{dev}")
    ok[starts[starts >= 0]] = True
    assert bool(ok.all()), "segmented output not sorted"
    del o, ok
    looped()  # warm-up of the per-array path
    lms, llaunch = [], 0
    for _ in range(2):
        ms, llaunch = looped()
        lms.append(ms)
    assert torch.equal(work, out_b), "batched and per-array results differ"
    del out_b, work, pristine
    b_ms = sum(bms) / len(bms)
    l_ms = sum(lms) / len(lms)
    cpu = None
    if with_cpu and not args.no_cpu:
        import multiprocessing as mp
        import oracle

        oracle.build()
        kw = dict(fanout=p.fanout, basecase_threshold=p.basecase_threshold, sample_rate=p.sample_rate,
                  recurse_model=p.recurse_model)
        pick = list(range(0, nseg, max(1, nseg // 48)))[:48]
        segs = [keys[int(off[s]):int(off[s + 1])] for s in pick]
        nk = sum(x.size for x in segs)
        t0 = time.perf_counter()
        for x in segs:
            assert _oracle_segments((x, kw)) == 0
        t1 = time.perf_counter() - t0
        cores = os.cpu_count() or 1
        with mp.get_context("spawn").Pool(cores) as pool:
            t0 = time.perf_counter()
            assert all(r == 0 for r in pool.map(_oracle_segments, [(x, kw) for x in segs]))
            tm = time.perf_counter() - t0
        cpu = {"value": nk / t1, "unit": "keys/s", "cores": 1, "kind": "oracle",
               "sample": f"{len(segs)} of the {nseg} segments ({nk} keys), one thread",
               "all_cores": {"value": nk / tm, "cores": cores, "note": "same segments, spawn pool, one per task"}}
    return {
        "workload": f"C4: {nseg} float64 segments, lengths log-uniform in [1e3, 1e6] ({n} keys), "
                    "distribution per segment from the six of C2, shift U[-1e3,1e3], scale log-U[1e-3,1e3]",
        "keys": n, "batched": {"value": n / (b_ms / 1e3), "unit": "keys/s", "ms": b_ms,
                               "gpu_launches": int(bst.kernel_launches)},
        "per_array_calls": {"value": n / (l_ms / 1e3), "unit": "keys/s", "ms": l_ms, "gpu_launches": llaunch},
        "batched_speedup": l_ms / b_ms,
        "params": {"fanout": p.fanout, "basecase_threshold": p.basecase_threshold, "sample_rate": p.sample_rate,
                   "recurse_model": p.recurse_model,
                   "chosen_by": f"ls_autotune_segmented on the first {tseg} segments ({int(off[tseg])} keys); "
                                f"{rep.configs} configurations, {rep.base_ms:.3f} -> {rep.best_ms:.3f} ms"},
        "cpu_baseline": cpu, "clocks": clk.summary(), "l2": "4.7 GB of keys, larger than L2; no flush",
    }


def c5_measure(lsg, ctx, args, torch, stream):
    """C5: 2e9 skewed uint64 keys (16 GB), RETRAIN recursion (a new sample and
    model per bucket), learned partitioner against the splitter tree on the
    same kernels, with per-pass achieved bandwidth."""
    dev = 0
    n = int(args.c5_n)
    pristine = datagen.skewed_u64_device(n, 5, f"cuda:{dev}").view(torch.int64)
    work = torch.empty_like(pristine)
    peak, _ = measured_peak()
    out = {"workload": f"C5: {n} uint64 keys (piecewise-linear CDF over 64 Dirichlet(0.3) pieces + 1% in 100 "
                       "lognormal(sigma=2) clusters), RETRAIN recursion, T = 4096",
           "keys": n, "l2": "16 GB of keys, larger than L2; no flush"}
    for name, part in (("learned", lsg.LS_PART_AUTO), ("splitter", lsg.LS_PART_SPLITTER)):
        p = lsg.ls_params_default(flags=lsg.LS_FLAG_TIME_PASSES, basecase_threshold=BASECASE_T,
                                  recurse_model=lsg.LS_RECURSE_RETRAIN, partitioner=part)
        ctx.workspace(n, 1, lsg.LS_U64, p)
        ms, sts = [], []
        for step in range(3):  # one warm-up, two timed
            work.copy_(pristine)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = lsg.ls_sort(ctx, work, p, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if step:
                ms.append(e0.elapsed_time(e1))
                sts.append(st)
        w = work.view(torch.int64)
        o = w ^ (-(2**63))  # u64 order as signed
        assert bool((o[1:] >= o[:-1]).all()), "C5 output not sorted"
        del o
        passes = {}
        for st in sts:
            for k, v in st.passes().items():
                a = passes.setdefault(k, {"ms": 0.0, "keys": 0})
                a["ms"] += v["ms"] / len(sts)
                a["keys"] += v["keys"] / len(sts)
        frac = {}
        for k, per_key in (("scatter", SCATTER_BYTES_PER_KEY), ("classify", CLASSIFY_BYTES_PER_KEY),
                           ("base", SCATTER_BYTES_PER_KEY)):
            if k in passes and passes[k]["ms"] > 0:
                gbs = per_key * passes[k]["keys"] / (passes[k]["ms"] / 1e3) / 1e9
                frac[k] = {"gbs": gbs, "frac": gbs / peak}
        m = sum(ms) / len(ms)
        out[name] = {"value": n / (m / 1e3), "unit": "keys/s", "ms": m,
                     "root_decision": int(sts[-1].root_decision), "levels": int(sts[-1].levels_used),
                     "level1_max_bucket": int(sts[-1].level[0].max_child),
                     "passes_ms": {k: v["ms"] for k, v in passes.items()}, "pass_roofline": frac}
        ctx.free_workspace()
    out["learned_speedup"] = out["splitter"]["ms"] / out["learned"]["ms"]
    del work, pristine
    return out


def run_c4(args):
    """The C4 line alone (--workload c4)."""
    import torch

    rank, world, local = dist_env()
    if world > 1 and rank != 0:
        return 0
    dev = 0
    torch.cuda.set_device(dev)
    import paper_2307_08637_gb300 as lsg

    stream = torch.cuda.current_stream()
    ctx = lsg.Context(dev)
    r = c4_measure(lsg, ctx, args, torch, stream)
    line = {
        "metric": "keys/s, batched segmented sort vs one ls_sort call per array (4096 f64 segments), 1 GB300",
        "value": r["batched"]["value"], "unit": "keys/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": r["batched"]["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": r["workload"], "params": r["params"], "l2": r["l2"]},
        "per_array_calls": r["per_array_calls"], "batched_speedup": r["batched_speedup"],
        "gpu_launches": r["batched"]["gpu_launches"], "cpu_baseline": r["cpu_baseline"], "clocks": r["clocks"],
    }
    ctx.close()
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c4":
        return run_c4(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
