"""The benchmark's multi-rank plumbing on CPU (gloo, world size 2): barrier
and max-over-ranks of the per-rank times, rank 0 alone printing, and the
reference arm run by rank 0 only.  The simulator itself is replicas only: (time,
frequency) instances are independent, so ranks share no data."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


CHILD = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import bench
rank, world, local = bench.dist_env()
d = bench.Dist(world)
d.barrier()
t = d.max(1.5 + rank)       # rank 1 is slower: the job time is its time
d.barrier()
d.close()
print(json.dumps({{"rank": rank, "world": world, "max": t}}))
"""


def run_ranks(code: str, world: int = 2, timeout: int = 120):
    port = free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=timeout)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_barrier_and_max_over_two_gloo_ranks():
    outs = run_ranks(CHILD.format(root=ROOT))
    lines = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert sorted(l["rank"] for l in lines) == [0, 1]
    assert all(l["world"] == 2 and l["max"] == 2.5 for l in lines)


def test_reference_arm_runs_on_rank_zero_only():
    pytest.importorskip("numpy")
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); sys.argv = ['bench.py', '--impl', 'reference', "
            "'--small', '--steps', '1', '--warmup', '0', '--gpus', '2']; import bench; bench.main()")
    outs = run_ranks(code, timeout=600)
    printed = [o for o in outs if o.strip()]
    assert len(printed) == 1
    line = json.loads(printed[0].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
