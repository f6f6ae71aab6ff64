"""bench.py's multi-rank host logic with two gloo ranks on the CPU: both
ranks agree on the slowest rank's step time, every rank sorts its own
inputs (weak scaling, no collective on the data path), the whole-job value
counts every rank's keys, and the reference arm prints exactly one line,
from rank 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _torchrun(args, timeout):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port())] + args
    env = dict(os.environ, OMP_NUM_THREADS="1")
    return subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout, env=env)


def _json_lines(out):
    return [json.loads(line) for line in out.splitlines() if line.startswith("{")]


def test_two_ranks_agree_on_the_slowest_step_and_use_their_own_inputs():
    r = _torchrun([os.path.join("tests", "rank_worker.py")], 300)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = _json_lines(r.stdout)
    assert sorted(d["rank"] for d in lines) == [0, 1]
    for d in lines:
        assert d["world"] == 2
        assert d["max_ms"] == 15.0
        assert len(set(d["seeds"])) == 2
        assert d["value"] == pytest.approx(2 * 1000 / 0.015)


def test_reference_arm_prints_one_line_under_two_ranks():
    r = _torchrun(["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"], 600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
