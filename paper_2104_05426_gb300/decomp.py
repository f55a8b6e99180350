"""Source/observation (S-O) decomposition of one field evaluation.

The paper scales past one GPU by cutting the source and the observation
regions into rectangular sub-boxes and evaluating every pair of a source box
and an observation box on its own, one pair per GPU (Sec. 2.2, Fig. 2): the
observation boxes are independent, and the fields of the pairs that share an
observation box add up.

Here:

* the source grid is cut along whole bricks by ``jefi_so_partition``; a
  box's handle keeps the whole grid's lattice (``src_origin``), so its cell
  centres, distances and retarded slots are bit-identical to the whole
  problem's, and it pushes its slices straight from the whole grid's arrays
  (``jefi_push_sources_region``);
* the observation points are cut into contiguous chunks of whole 256-point
  tiles;
* pair p = (chunk o, box k), p = o * n_boxes + k, belongs to rank p mod world;
* the fields of a chunk are the FP64 sum of its pairs in box order
  (``jefi_sum_fields``), the same on one rank or many: an observation split
  needs no exchange at all, a source split one gather of the pairs' fields.

Every sum runs in libjefi's kernels; this module does host bookkeeping and,
across ranks, one ``all_gather`` of the pairs' fields (torch.distributed).
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import (Handle, default_params, jefi_create, jefi_destroy, jefi_eval_fields,
               jefi_get_info, jefi_push_sources_region, jefi_so_partition, jefi_sum_fields)

TILE = 256


def obs_chunks(n_obs: int, parts: int) -> List[Tuple[int, int]]:
    """[begin, end) of `parts` contiguous chunks of whole 256-point tiles
    (the last chunk takes the ragged tail; a chunk may be empty)."""
    if parts < 1:
        raise ValueError("parts must be positive")
    n_tiles = (n_obs + TILE - 1) // TILE
    out = []
    for k in range(parts):
        t0, t1 = k * n_tiles // parts, (k + 1) * n_tiles // parts
        out.append((min(t0 * TILE, n_obs), min(t1 * TILE, n_obs)))
    return out


def pair_owner(p: int, world: int) -> int:
    return p % world


class SODecomposition:
    """The S-O pairs of one problem owned by one rank.

    src       the whole source grid (jefi_grid)
    obs       [N, 3] float64 observation points (host)
    params    keyword arguments of default_params (c, dt, t0, history_slots, precision, ...)
    src_parts (px, py, pz) source boxes; obs_parts observation chunks
    rank, world   this rank and the number of ranks (pairs are dealt round robin)
    """

    def __init__(self, src, obs: np.ndarray, params: dict, src_parts: Sequence[int] = (1, 1, 1),
                 obs_parts: int = 1, rank: int = 0, world: int = 1, torch_allocator: bool = False):
        self.src = src
        self.full_n = tuple(int(src.n[a]) for a in range(3))
        self.obs = np.ascontiguousarray(obs, dtype=np.float64).reshape(-1, 3)
        self.boxes = jefi_so_partition(src, src_parts)
        self.chunks = obs_chunks(len(self.obs), obs_parts)
        self.rank, self.world = rank, world
        self.pairs = [(o, k) for o in range(len(self.chunks)) for k in range(len(self.boxes))]
        self.mine = [p for p in range(len(self.pairs)) if pair_owner(p, world) == rank]
        self.handles: Dict[int, Handle] = {}
        for p in self.mine:
            o, k = self.pairs[p]
            sub, origin = self.boxes[k]
            b0, b1 = self.chunks[o]
            kw = dict(params)
            kw["src_origin"] = origin
            prm = default_params(**kw)
            self.handles[p] = jefi_create(sub, obs_points=self.obs[b0:b1], params=prm,
                                          torch_allocator=torch_allocator)

    def valid_window(self):
        """Times at which every pair of this rank can be evaluated: the
        intersection of the pairs' windows (each box sees its own range of
        distances, so its window differs)."""
        from . import jefi_valid_window

        lo, hi = -np.inf, np.inf
        for h in self.handles.values():
            a, b = jefi_valid_window(h)
            lo, hi = max(lo, a), min(hi, b)
        return lo, hi

    def push(self, rho, J, drho_dt=None, dJ_dt=None, stream=None):
        """One slice of the whole grid (x fastest): every owned pair takes its box."""
        for p, h in self.handles.items():
            _, k = self.pairs[p]
            jefi_push_sources_region(h, rho, J, self.full_n, self.boxes[k][1], drho_dt, dJ_dt, stream=stream)

    def evaluate_pairs(self, t: float, stream=None) -> Dict[int, tuple]:
        """E and B ([n_chunk, 3] CUDA float64) of every owned pair at time t."""
        import torch

        out = {}
        for p, h in self.handles.items():
            o, _ = self.pairs[p]
            n = self.chunks[o][1] - self.chunks[o][0]
            E = torch.empty((n, 3), dtype=torch.float64, device="cuda")
            B = torch.empty_like(E)
            if n > 0:
                jefi_eval_fields(h, t, E, B, stream=stream)
            out[p] = (E, B)
        return out

    def fields(self, t: float, group=None, stream=None):
        """E and B at every observation point ([N, 3] CUDA float64), the same on
        every rank: the pairs' fields gathered (world > 1) and summed per chunk
        in box order."""
        import torch

        local = self.evaluate_pairs(t, stream=stream)
        every = gather_pair_fields(local, self.pairs, self.chunks, self.world, self.rank, group)
        E = torch.empty((len(self.obs), 3), dtype=torch.float64, device="cuda")
        B = torch.empty_like(E)
        nb = len(self.boxes)
        for o, (b0, b1) in enumerate(self.chunks):
            if b1 == b0:
                continue
            parts = [every[o * nb + k] for k in range(nb)]
            jefi_sum_fields([x[0] for x in parts], [x[1] for x in parts], E[b0:b1], B[b0:b1], stream=stream)
        return E, B

    def device_bytes(self) -> int:
        return sum(jefi_get_info(h)["device_bytes"] for h in self.handles.values())

    def close(self):
        for h in self.handles.values():
            jefi_destroy(h)
        self.handles = {}


def gather_pair_fields(local: Dict[int, tuple], pairs, chunks, world: int, rank: int, group=None,
                       device=None) -> Dict[int, tuple]:
    """Every pair's (E, B) on every rank: with one rank the local dict; else
    one all_gather of each rank's pairs (stacked and padded to the longest
    chunk) through torch.distributed, unpacked by owner.  No arithmetic: the
    sums are the caller's (in box order).  `device`: where the gathered
    tensors live (default: the local tensors' device, else CUDA)."""
    if world == 1:
        return dict(local)
    import torch
    import torch.distributed as dist

    n_pairs = len(pairs)
    per_rank = [[p for p in range(n_pairs) if pair_owner(p, world) == r] for r in range(world)]
    slots = max(len(x) for x in per_rank)
    longest = max((b1 - b0 for b0, b1 in chunks), default=0)
    if device is None:
        any_t = next(iter(local.values()))[0] if local else None
        device = any_t.device if any_t is not None else torch.device("cuda")
    mine = torch.zeros((max(slots, 1), 2, max(longest, 1), 3), dtype=torch.float64, device=device)
    for i, p in enumerate(per_rank[rank]):
        E, B = local[p]
        n = E.shape[0]
        mine[i, 0, :n] = E
        mine[i, 1, :n] = B
    got = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(got, mine, group=group)
    out = {}
    for r in range(world):
        for i, p in enumerate(per_rank[r]):
            o, _ = pairs[p]
            n = chunks[o][1] - chunks[o][0]
            out[p] = (got[r][i, 0, :n].contiguous(), got[r][i, 1, :n].contiguous())
    return out
