"""S-O decomposition across ranks, host side, on CPU (gloo, world size 2).

The paper runs one S-O pair (a source box with an observation box) per GPU
and adds the fields of the pairs that share an observation box (Sec. 2.2,
Fig. 2).  Checked here without a GPU: the brick-aligned source partition
covers every cell exactly once; the observation chunks cover every point;
and two ranks, each holding one source half, exchange their pairs' fields
with the library's gather, whose box-ordered sum equals the single-rank
result.  The pairs' fields come from the FP64 oracle (the per-pair GPU
evaluation and the device sum are the GPU tests' part)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np

import paper_2104_05426_gb300 as jefi
from paper_2104_05426_gb300.decomp import obs_chunks, pair_owner

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_partition_covers_every_cell_once():
    for n, parts in (((10, 9, 17), (2, 1, 3)), ((4, 4, 4), (3, 1, 1)), ((33, 7, 1), (4, 2, 1))):
        g = jefi.grid(n, (0.1, -0.2, 0.3), (0.05, 0.07, 0.11))
        boxes = jefi.jefi_so_partition(g, parts)
        assert len(boxes) == parts[0] * parts[1] * parts[2]
        seen = np.zeros(n[::-1], dtype=np.int32)
        for sub, org in boxes:
            assert tuple(sub.lo) == tuple(g.lo) and tuple(sub.d) == tuple(g.d)
            assert all(o % 4 == 0 for o in org)             # boxes start on whole bricks
            seen[org[2]:org[2] + sub.n[2], org[1]:org[1] + sub.n[1], org[0]:org[0] + sub.n[0]] += 1
        assert (seen == 1).all()
    for n_obs, parts in ((1000, 3), (256, 4), (0, 2), (4097, 2)):
        ch = obs_chunks(n_obs, parts)
        assert ch[0][0] == 0 and ch[-1][1] == n_obs
        assert all(a[1] == b[0] for a, b in zip(ch, ch[1:]))
        assert all(b0 % 256 == 0 for b0, _ in ch)


WORKER = r"""
import sys, json
sys.path.insert(0, {root!r})
import numpy as np
import torch
import torch.distributed as dist
import bench
import oracle
import paper_2104_05426_gb300 as jefi
from paper_2104_05426_gb300.decomp import gather_pair_fields, obs_chunks, pair_owner
world, rank, _ = bench.dist_env()
bench.init_dist(world, "gloo")
# dyadic lattice: a sub-box's own grid (lo + origin d) has bit-identical centres
n, lo, d = (12, 8, 8), (-0.75, -0.5, -0.5), (0.125, 0.125, 0.125)
src = jefi.grid(n, lo, d)
rng = np.random.Generator(np.random.PCG64(3))
obs = rng.uniform(-1.5, 1.5, (600, 3))
dt, H, t = 0.0625, 64, 3.0
rho = rng.standard_normal((H, n[0] * n[1] * n[2]))
J = rng.standard_normal((H, n[0] * n[1] * n[2], 3))
boxes = jefi.jefi_so_partition(src, (2, 1, 1))
chunks = obs_chunks(len(obs), 2)
pairs = [(o, k) for o in range(len(chunks)) for k in range(len(boxes))]
local = {{}}
for p, (o, k) in enumerate(pairs):
    if pair_owner(p, world) != rank:
        continue
    sub, org = boxes[k]
    m = [sub.n[a] for a in range(3)]
    r4 = rho.reshape(H, n[2], n[1], n[0])[:, org[2]:org[2] + m[2], org[1]:org[1] + m[1], org[0]:org[0] + m[0]]
    j4 = J.reshape(H, n[2], n[1], n[0], 3)[:, org[2]:org[2] + m[2], org[1]:org[1] + m[1], org[0]:org[0] + m[0]]
    b0, b1 = chunks[o]
    E, B = oracle.fields(m, [lo[a] + org[a] * d[a] for a in range(3)], d, obs[b0:b1],
                         np.ascontiguousarray(r4.reshape(H, -1)), np.ascontiguousarray(j4.reshape(H, -1, 3)),
                         dt=dt, t=t)
    local[p] = (torch.from_numpy(E), torch.from_numpy(B))
every = gather_pair_fields(local, pairs, chunks, world, rank, device=torch.device("cpu"))
E = np.zeros((len(obs), 3)); B = np.zeros((len(obs), 3))
for o, (b0, b1) in enumerate(chunks):
    for k in range(len(boxes)):                      # box order
        E[b0:b1] += every[o * len(boxes) + k][0].numpy()
        B[b0:b1] += every[o * len(boxes) + k][1].numpy()
Ew, Bw = oracle.fields(n, lo, d, obs, rho, J, dt=dt, t=t)
eE = float(np.linalg.norm(E - Ew) / np.linalg.norm(Ew)); eB = float(np.linalg.norm(B - Bw) / np.linalg.norm(Bw))
print(json.dumps({{"rank": rank, "owned": sorted(local), "eE": eE, "eB": eB, "E0": E[:2].tolist()}}))
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_ranks_gather_source_halves_in_box_order():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(r), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    res = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err
        res.append(json.loads(out.strip().splitlines()[-1]))
    # pairs dealt round robin: 2 chunks x 2 source boxes over 2 ranks
    assert res[0]["owned"] == [0, 2] and res[1]["owned"] == [1, 3]
    for r in res:
        assert r["eE"] <= 1e-12 and r["eB"] <= 1e-12
    assert res[0]["E0"] == res[1]["E0"]           # every rank ends with the same fields, bit for bit
