"""Multi-rank host logic on CPU (gloo, world size 2): the timing reduction
(max over ranks), barriers, weak-scaling sharding and the reference arm's
rank-0-only rule.  The data path has no collective; only these host steps
use torch.distributed."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import bench
d = bench.Dist(want_cuda=False)
r = d.rank
out = {{"rank": r, "world": d.world, "max": d.max(10.0 + r), "sum": d.sum(1.0 + r)}}
d.barrier()
print(json.dumps(out))
d.close()
"""


def _launch(code_or_args, world=2, timeout=120):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="2")
        cmd = [sys.executable, "-c", code_or_args] if isinstance(code_or_args, str) else [sys.executable] + code_or_args
        procs.append(subprocess.Popen(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                                      cwd=ROOT))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=timeout)
        assert p.returncode == 0, e
        outs.append(o)
    return outs


def test_max_and_sum_over_two_ranks():
    outs = _launch(WORKER.format(root=ROOT))
    rows = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert sorted(r["rank"] for r in rows) == [0, 1]
    for r in rows:
        assert r["world"] == 2 and r["max"] == 11.0 and r["sum"] == 3.0


def test_reference_arm_prints_once_on_rank_zero():
    outs = _launch(["bench.py", "--impl", "reference", "--workload", "tiny", "--steps", "1", "--warmup", "0",
                    "--gpus", "2"], timeout=300)
    lines = [o.strip() for o in outs if o.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0].splitlines()[-1])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_single_process():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "tiny", "--steps", "2",
                          "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=300,
                         env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert out.returncode == 0, out.stderr
    d = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
