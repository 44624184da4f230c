"""The multi-rank host logic of bench.py on CPU: two gloo ranks on 127.0.0.1
(no GPU).  Covers the rank set-up, the barrier, the max-over-ranks reduction
of the timed region, and the reference arm's rule that rank 0 alone runs and
prints while the other ranks exit 0 without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys, types
sys.path.insert(0, {root!r})
import bench
ws, rank, local = bench.dist_setup()
assert ws == 2 and rank == int(os.environ["RANK"])
bench.barrier(ws)
# each rank times a different region; the reported time is the largest
got = bench.max_over_ranks(1.5 + rank, ws)
assert got == 2.5, got
if {reference}:
    args = types.SimpleNamespace(steps=1, warmup=0, gpus=2, workload="bipoles40_256x256x256")
    bench.run_reference(args, ws, rank)
import torch.distributed as dist
dist.destroy_process_group()
print("rank-done", rank, flush=True)
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_two(reference):
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(r),
                   LOCAL_RANK=str(r), CUDA_VISIBLE_DEVICES="")
        code = CHILD.format(root=ROOT, reference=bool(reference))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, cwd=ROOT, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=300)
        except subprocess.TimeoutExpired:
            p.kill()
            o, e = p.communicate()
        outs.append((p.returncode, o, e))
    return outs


def test_two_ranks_barrier_and_max():
    pytest.importorskip("torch")
    outs = _run_two(reference=False)
    for r, (rc, o, e) in enumerate(outs):
        assert rc == 0, e[-2000:]
        assert f"rank-done {r}" in o


def test_reference_arm_rank0_only():
    pytest.importorskip("torch")
    outs = _run_two(reference=True)
    lines = []
    for r, (rc, o, e) in enumerate(outs):
        assert rc == 0, e[-2000:]
        js = [ln for ln in o.splitlines() if ln.startswith("{")]
        lines.append(js)
    assert len(lines[0]) == 1 and lines[1] == []
    d = json.loads(lines[0][0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
