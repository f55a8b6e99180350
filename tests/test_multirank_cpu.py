"""World-size-2 gloo checks of the benchmark's multi-rank host logic: the
replicas-only path takes the maximum step time over ranks and only rank 0
reports.  The reference arm runs on rank 0 alone."""
import os
import socket
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
world, rank, local = bench.dist_env()
bench.init_dist(world, "gloo")
local_ms = 10.0 * (rank + 1)
m = bench.max_over_ranks(local_ms, world)
bench.barrier(world)
print(json.dumps({{"rank": rank, "max": m}}))
dist.destroy_process_group()
"""


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def launch(code, world=2):
    port = free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, WORLD_SIZE=str(world), RANK=str(r), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(out)
    return outs


def test_max_over_ranks_gloo():
    import json

    outs = launch(WORKER.format(root=ROOT))
    vals = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    assert all(v["max"] == 20.0 for v in vals)


def test_reference_arm_non_zero_ranks_exit_quietly():
    code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench; "
            "bench.main(['--impl', 'reference', '--steps', '1', '--warmup', '3'])")
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
