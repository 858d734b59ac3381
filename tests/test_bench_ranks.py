"""The multi-rank parts of bench.py on CPU: replicas launched as world_size-2 gloo
ranks combine their timings as the maximum over ranks, the job throughput counts
every rank's replica, and the reference arm runs on rank 0 only."""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys, json
sys.path.insert(0, %r)
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
t = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
m = bench.job_mlups(1000, 10, world, t)
print(json.dumps({"rank": rank, "t": t, "mlups": m}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _launch(code, world=2, extra_env=None):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(r),
                   WORLD_SIZE=str(world), LOCAL_RANK=str(r))
        env.update(extra_env or {})
        procs.append(subprocess.Popen([sys.executable, "-c", code] if isinstance(code, str) else code,
                                      env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True, cwd=ROOT))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_max_over_ranks_and_job_throughput_gloo():
    pytest.importorskip("torch")
    outs = _launch(CHILD % ROOT)
    res = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert [r["t"] for r in res] == [15.0, 15.0]
    # 1000 fluid nodes x 10 steps x 2 replicas in 15 ms
    assert all(abs(r["mlups"] - 1000 * 10 * 2 / 15e-3 / 1e6) < 1e-12 for r in res)


def test_reference_arm_prints_on_rank_zero_only():
    outs = _launch([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                    "--steps", "1", "--warmup", "3", "--gpus", "2"])
    lines = [o.strip() for o in outs]
    assert lines[1] == ""
    line = json.loads(lines[0].splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
