"""Continuous-batching serving loop for field-evaluation requests.

A request asks for E and B on an observation grid at a time t, against one of
several source problems whose histories stay resident on the GPU (the paper
keeps rho and J on the device between calls, Sec. 2.2; here many problems and
many requests share the device).  The loop:

* keeps one base handle per source problem (FP32 compensated ring, sized for
  views of any staged band) and pushes one new slice to every problem per
  tick, generated on the device;
* serves each request through an observation view of its problem (cached per
  observation grid; a view is never in two batches at once);
* admits arrived requests first-in first-out while the device memory of their
  views and outputs fits the budget;
* launches admitted requests as they come, as one jefi_eval_batch per stream,
  on a small pool of streams, so batches that arrive while others run are
  admitted and overlap them on the device (continuous batching);
* orders every slice push after the in-flight batches that read the same ring
  and every later batch after that push (CUDA events);
* records arrival, launch and completion times; latency = completion - arrival.

Every step of the field evaluation runs in libjefi's kernels; this module is
host-side scheduling only.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

from workloads import OscBlob, OscillatingGaussians

from . import (JEFI_EEVICTED, JEFI_FLAG_SHARED_RING, JefiError, default_params, grid, jefi_batch_plan_create,
               jefi_batch_plan_destroy, jefi_batch_plan_launch, jefi_batch_plan_tune, jefi_create,
               jefi_create_view, jefi_destroy, jefi_eval_batch, jefi_get_info, jefi_push_sources,
               jefi_valid_window)


class ServedProblem:
    """A resident source problem: a cube grid of Gaussian charges on bounded
    oscillating paths (the seeded source model of ``workloads``: the charges
    stay in the box however long the loop runs), its base handle and a
    device-side slice generator."""

    def __init__(self, side: int, half_width: float, H: int, dt: float, blobs: List[OscBlob],
                 device="cuda", stream=None):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.side = side
        self.L = half_width
        self.H = H
        self.dt = dt
        self.blobs = blobs
        self.model = OscillatingGaussians(blobs)
        d = 2.0 * half_width / side
        self.grid = grid((side,) * 3, (-half_width,) * 3, (d,) * 3)
        prm = default_params(dt=dt, history_slots=H, precision="fp32c", flags=JEFI_FLAG_SHARED_RING)
        # PyTorch's caching allocator: views created and destroyed while the
        # loop runs then cost no cudaMalloc / cudaFree (cudaFree waits for the device)
        self.handle = jefi_create(self.grid, obs_points=np.zeros((0, 3)), params=prm, stream=stream,
                                  torch_allocator=True)
        # cell centres resident on the device: a slice is generated by device
        # ops alone (a host-to-device copy per slice would block the host
        # behind the push stream, which waits for the batches in flight)
        ax = -half_width + (torch.arange(side, dtype=torch.float64, device=self.device) + 0.5) * d
        z, y, x = torch.meshgrid(ax, ax, ax, indexing="ij")
        self.pts = torch.stack([x.reshape(-1), y.reshape(-1), z.reshape(-1)], dim=1)
        self.n_pushed = 0
        self.last_push = None               # event after the latest push
        self.readers: List = []             # events of batches reading the ring

    def slice_at(self, t: float):
        """rho = sum of the blobs' Gaussians at time t, J = sum of rho_blob v_blob."""
        rho, J = self.model.sample_torch(self.pts, t)
        return rho.contiguous(), J.contiguous()

    def push_next(self, stream):
        """Push the next slice on `stream` after every batch still reading the ring."""
        torch = self.torch
        for ev in self.readers:
            stream.wait_event(ev)
        self.readers = []
        with torch.cuda.stream(stream):
            rho, J = self.slice_at(self.n_pushed * self.dt)
            jefi_push_sources(self.handle, rho, J, stream=stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.last_push = ev
        self.n_pushed += 1


class SliceBatch:
    """The next slice of many served problems at once, by the formula of
    ``OscillatingGaussians.sample_torch`` (rho = sum q G(r - c(t)), J = sum
    q G(r - c(t)) c'(t), blobs in order), with a few device operations per
    blob slot for all problems together instead of a dozen per blob per
    problem: the serving loop pushes to every problem every tick, and its
    single host thread would otherwise spend most of a tick launching the
    generator's small kernels.  Problems with fewer blobs carry zero-charge
    blobs (they add exact zeros).  `pts` of each problem on one device."""

    def __init__(self, problems):
        import torch

        self.torch = torch
        self.problems = list(problems)
        dev = self.problems[0].pts.device
        self.counts = [p.pts.shape[0] for p in self.problems]
        self.offsets = np.concatenate([[0], np.cumsum(self.counts)]).astype(np.int64)
        self.pts = torch.cat([p.pts for p in self.problems], dim=0)
        self.pidx = torch.repeat_interleave(torch.arange(len(self.problems), device=dev),
                                            torch.tensor(self.counts, device=dev))
        self.nb = max(len(p.blobs) for p in self.problems)
        P, B = len(self.problems), self.nb
        sig = np.ones((P, B, 3))
        coef = np.zeros((P, B))
        for i, p in enumerate(self.problems):
            for k, b in enumerate(p.blobs):
                sig[i, k] = b.sigma
                coef[i, k] = b.q * (1.0 / ((2.0 * math.pi) ** 1.5 * b.sigma[0] * b.sigma[1] * b.sigma[2]))
        self.sig = torch.tensor(sig, dtype=torch.float64, device=dev)
        self.coef = torch.tensor(coef, dtype=torch.float64, device=dev)

    def sample(self, times):
        """rho [N_total] and J [N_total, 3] of every problem at its time
        (times[i] for problem i); problem i's rows start at offsets[i]."""
        torch = self.torch
        P, B = len(self.problems), self.nb
        cv = np.zeros((2, P, B, 3))
        for i, p in enumerate(self.problems):
            for k, b in enumerate(p.blobs):
                c, v = p.model._centre(b, times[i])
                cv[0, i, k] = c
                cv[1, i, k] = v
        cv = torch.from_numpy(cv)
        if self.pts.is_cuda:   # pinned and asynchronous: the host does not wait for the stream
            cv = cv.pin_memory().to(self.pts.device, non_blocking=True)
        rho = torch.zeros(self.pts.shape[0], dtype=torch.float64, device=self.pts.device)
        J = torch.zeros((self.pts.shape[0], 3), dtype=torch.float64, device=self.pts.device)
        for k in range(B):
            u = (self.pts - cv[0, :, k][self.pidx]) / self.sig[:, k][self.pidx]
            g = self.coef[:, k][self.pidx] * torch.exp(-0.5 * (u * u).sum(dim=1))
            rho += g
            J += g[:, None] * cv[1, :, k][self.pidx]
        return rho, J


@dataclass
class Request:
    rid: int
    problem: int
    obs_side: int
    frac: float                      # position of t inside the valid window
    arrival: float                   # seconds after the start of the run
    t: float = math.nan
    launch: float = math.nan
    done: float = math.nan
    error: int = 0
    E: object = None
    B: object = None
    view: object = None
    pairs: int = 0


@dataclass
class ServingStats:
    completed: int
    rejected: int
    evicted: int
    failed: int
    wall_s: float
    p50_ms: float
    p99_ms: float
    mean_ms: float
    requests_per_s: float
    pairs_per_s: float
    max_batch: int
    mean_batch: float
    peak_bytes: int
    views_created: int
    latencies_ms: List[float] = field(default_factory=list)

    def as_dict(self):
        d = dict(self.__dict__)
        d.pop("latencies_ms")
        return d


class ServingEngine:
    def __init__(self, problems: List[ServedProblem], obs_half_width: float, n_streams: int = 4,
                 memory_budget: float = 64e9, max_batch: int = 64, tick_s: Optional[float] = None,
                 keep_outputs: bool = False, keep_ids=None):
        import torch

        self.torch = torch
        self.problems = problems
        self.obs_half_width = obs_half_width
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.push_stream = torch.cuda.Stream()
        self.gen_stream = torch.cuda.Stream()   # slice generation, apart from the batches' order
        self.slices = SliceBatch(problems)
        self.memory_budget = memory_budget
        self.max_batch = max_batch
        self.tick_s = tick_s
        self.keep_outputs = keep_outputs
        self.keep_ids = set(keep_ids or ())     # request ids whose E and B are kept
        self.views: Dict[Tuple[int, int], List] = {}     # (problem, side) -> [[view, busy, bytes]]
        self.view_bytes: Dict[Tuple[int, int], int] = {}  # measured device bytes of a view
        self.resident_bytes = sum(jefi_get_info(p.handle)["device_bytes"] for p in problems)
        self.used_bytes = self.resident_bytes
        self.peak_bytes = self.used_bytes
        self.views_created = 0

    # ------------------------------------------------------------------ pushes
    def _push_all(self):
        """One tick: the next slice of every problem, generated together on a
        stream of its own (it does not wait for the batches in flight), then
        pushed on the push stream, each problem's push after the batches still
        reading its ring; later batches wait for the push (last_push)."""
        torch = self.torch
        with torch.cuda.stream(self.gen_stream):
            rho, J = self.slices.sample([p.n_pushed * p.dt for p in self.problems])
            gen_done = torch.cuda.Event()
            gen_done.record(self.gen_stream)
        s = self.push_stream
        rho.record_stream(s)
        J.record_stream(s)
        s.wait_event(gen_done)
        off = self.slices.offsets
        for i, p in enumerate(self.problems):
            for ev in p.readers:
                s.wait_event(ev)
            p.readers = []
            jefi_push_sources(p.handle, rho[off[i]:off[i + 1]], J[off[i]:off[i + 1]], stream=s)
            ev = torch.cuda.Event()
            ev.record(s)
            p.last_push = ev
            p.n_pushed += 1

    # ------------------------------------------------------------------ views
    def _free_view(self, key):
        for entry in self.views.get(key, []):
            if not entry[1]:
                return entry
        return None

    def _create_view(self, req: Request):
        p = self.problems[req.problem]
        s = req.obs_side
        d = 2.0 * self.obs_half_width / s
        g = grid((s,) * 3, (-self.obs_half_width,) * 3, (d,) * 3)
        view = jefi_create_view(p.handle, obs_grid=g)
        nbytes = jefi_get_info(view)["device_bytes"]
        self.view_bytes[(req.problem, s)] = nbytes
        self.views_created += 1
        return [view, True, nbytes]

    def _evict_idle(self, need: int):
        """Destroy cached views that no batch is using until `need` bytes are freed."""
        freed = 0
        for key in list(self.views.keys()):
            keep = []
            for e in self.views[key]:
                if freed < need and not e[1]:
                    jefi_destroy(e[0])
                    self.used_bytes -= e[2]
                    freed += e[2]
                else:
                    keep.append(e)
            self.views[key] = keep
            if freed >= need:
                break

    def _output_bytes(self, side):
        return side ** 3 * 6 * 8

    # ------------------------------------------------------------------ run
    def run(self, requests: List[Request]) -> ServingStats:
        torch = self.torch
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        queue: deque = deque()
        admitted: List[Request] = []
        inflight: List[Tuple[object, int, List[Request]]] = []
        free_streams = list(range(len(self.streams)))
        done: List[Request] = []
        batch_sizes: List[int] = []
        rejected = 0            # refused by the memory budget
        evicted = 0             # the time's slices were overwritten before the launch
        failed = 0              # other errors of a batch
        torch.cuda.synchronize()
        start = time.perf_counter()
        next_tick = self.tick_s if self.tick_s else math.inf
        while pending or queue or admitted or inflight:
            now = time.perf_counter() - start
            progressed = False
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
                progressed = True
            if now >= next_tick:
                self._push_all()
                next_tick += self.tick_s
                progressed = True
            # admission, first in first out, by device memory (a view's real
            # bytes once one of its kind has been created, else an estimate)
            while queue:
                req = queue[0]
                key = (req.problem, req.obs_side)
                entry = self._free_view(key)
                if entry is not None:
                    entry[1] = True              # reserved: the eviction below must not take it
                out_bytes = self._output_bytes(req.obs_side)
                need = out_bytes
                if entry is None:
                    need += self.view_bytes.get(key, self._estimate_view_bytes(req))
                if self.used_bytes + need > self.memory_budget:
                    self._evict_idle(self.used_bytes + need - self.memory_budget)
                if self.used_bytes + need > self.memory_budget:
                    if entry is not None:
                        entry[1] = False         # not admitted: the view is idle again
                    if not inflight and not admitted:
                        queue.popleft()          # can never fit: reject
                        req.error = -1
                        rejected += 1
                        progressed = True
                        continue
                    break
                if entry is None:
                    entry = self._create_view(req)
                    if self.used_bytes + entry[2] + out_bytes > self.memory_budget:
                        # the estimate was low: make room, or give the view back and wait
                        self._evict_idle(self.used_bytes + entry[2] + out_bytes - self.memory_budget)
                        if self.used_bytes + entry[2] + out_bytes > self.memory_budget:
                            jefi_destroy(entry[0])
                            if not inflight and not admitted:
                                queue.popleft()
                                req.error = -1
                                rejected += 1
                                progressed = True
                                continue
                            break
                    self.views.setdefault(key, []).append(entry)
                    self.used_bytes += entry[2]
                queue.popleft()
                req.view = entry
                req.E = torch.empty((req.obs_side ** 3, 3), dtype=torch.float64, device="cuda")
                req.B = torch.empty_like(req.E)
                self.used_bytes += out_bytes
                self.peak_bytes = max(self.peak_bytes, self.used_bytes)
                req.pairs = self.problems[req.problem].side ** 3 * req.obs_side ** 3
                admitted.append(req)
                progressed = True
            # launch: one batch per free stream.  A request's time is placed in
            # its problem's valid window now, after the pushes enqueued so far
            # (the batch waits for them): a push between admission and launch
            # moves the window.
            while admitted and free_streams:
                si = free_streams.pop()
                stream = self.streams[si]
                batch = admitted[: self.max_batch]
                del admitted[: len(batch)]
                for p_idx in {r.problem for r in batch}:
                    if self.problems[p_idx].last_push is not None:
                        stream.wait_event(self.problems[p_idx].last_push)
                for r in batch:
                    lo, hi = jefi_valid_window(r.view[0])
                    if not math.isfinite(lo):
                        lo = hi - 4 * self.problems[r.problem].dt
                    r.t = lo + (hi - lo) * r.frac
                t_launch = time.perf_counter() - start
                try:
                    jefi_eval_batch([r.view[0] for r in batch], [r.t for r in batch],
                                    [r.E for r in batch], [r.B for r in batch], stream=stream)
                except JefiError as e:
                    for r in batch:
                        r.error = e.code
                ev = torch.cuda.Event()
                ev.record(stream)
                for r in batch:
                    r.launch = t_launch
                    self.problems[r.problem].readers.append(ev)
                inflight.append((ev, si, batch))
                batch_sizes.append(len(batch))
                progressed = True
            # completion
            still = []
            for ev, si, batch in inflight:
                if ev.query():
                    t_done = time.perf_counter() - start
                    for r in batch:
                        r.done = t_done
                        r.view[1] = False
                        self.used_bytes -= self._output_bytes(r.obs_side)
                        if r.error == JEFI_EEVICTED:
                            evicted += 1
                        elif r.error:
                            failed += 1
                        else:
                            done.append(r)
                        if not (self.keep_outputs or r.rid in self.keep_ids):
                            r.E = r.B = None
                    free_streams.append(si)
                    progressed = True
                else:
                    still.append((ev, si, batch))
            inflight = still
            if not progressed:
                time.sleep(50e-6)
        wall = time.perf_counter() - start
        lat = sorted((r.done - r.arrival) * 1e3 for r in done)
        pairs = sum(r.pairs for r in done)

        def pct(q):
            if not lat:
                return math.nan
            return float(np.percentile(np.asarray(lat), q))

        return ServingStats(completed=len(done), rejected=rejected, evicted=evicted, failed=failed, wall_s=wall, p50_ms=pct(50),
                            p99_ms=pct(99), mean_ms=float(np.mean(lat)) if lat else math.nan,
                            requests_per_s=len(done) / wall, pairs_per_s=pairs / wall,
                            max_batch=max(batch_sizes) if batch_sizes else 0,
                            mean_batch=float(np.mean(batch_sizes)) if batch_sizes else 0.0,
                            peak_bytes=int(self.peak_bytes), views_created=self.views_created,
                            latencies_ms=lat)

    def _estimate_view_bytes(self, req: Request) -> int:
        # a generous guess, used until a view of this (problem, side) exists and
        # its real bytes are known: partial sums dominate (a view holds 2 time
        # slots x splits x 6 x points x 8 B, at most 32 MB); this counts 8 slots
        # and about two waves of (tile, split) items
        n = req.obs_side ** 3
        tiles = max(1, (n + 255) // 256)
        splits = max(1, min(608 // tiles, 64))
        return int(8 * splits * 6 * tiles * 256 * 8 + n * 3 * 8 * 2 + (1 << 20))

    def close(self):
        self.torch.cuda.synchronize()
        for entries in self.views.values():
            for e in entries:
                jefi_destroy(e[0])
        self.views = {}
        for p in self.problems:
            jefi_destroy(p.handle)


def make_problems(n: int, seed: int, sides=(16, 64), H_range=(64, 256), half_width=1.0,
                  obs_half_width=2.0, stream=None) -> List[ServedProblem]:
    """Seeded resident problems: cubic source grids over [-L,L]^3 with 1-4
    moving Gaussian charges; dt chosen so H slices just cover the pairs of an
    observation grid over [-2L,2L]^3.  Pushes H slices into each."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rng_path = np.random.Generator(np.random.PCG64([seed, 1]))   # path shapes, apart from the geometry draws
    out = []
    for _ in range(n):
        side = int(rng.integers(sides[0], sides[1] + 1))
        H = int(rng.integers(H_range[0], H_range[1] + 1))
        rmax = math.sqrt(3.0) * (half_width + obs_half_width)
        dt = rmax / (H - 8)
        blobs = []
        for _ in range(int(rng.integers(1, 5))):
            # speed up to 0.5c on a path of amplitude 0.2-0.5 around x0
            d = rng.standard_normal(3)
            d /= np.linalg.norm(d)
            speed = rng.uniform(0.0, 0.5)
            q = float(rng.choice([-1.0, 1.0]))
            sigma = float(rng.uniform(0.15, 0.35))
            x0 = rng.uniform(-0.2, 0.2, 3)
            amp = rng_path.uniform(0.2, 0.5)
            blobs.append(OscBlob(q, (sigma,) * 3, tuple(x0), tuple(amp * d), speed / amp,
                                 float(rng_path.uniform(0.0, 2.0 * math.pi))))
        p = ServedProblem(side, half_width, H, dt, blobs)
        out.append(p)
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    for p in out:
        for _ in range(p.H + 1):          # one past the ring: the oldest slice is evicted
            p.push_next(s)
    torch.cuda.synchronize()
    return out


def poisson_requests(n: int, rate: float, n_problems: int, obs_sides=(8, 48), seed: int = 7,
                     side_choices: Optional[List[int]] = None) -> List[Request]:
    """Seeded Poisson arrivals at `rate` per second; uniform problem, side and
    position in the valid window."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, n)
    arrivals = np.cumsum(gaps)
    reqs = []
    for i in range(n):
        if side_choices:
            side = int(side_choices[int(rng.integers(0, len(side_choices)))])
        else:
            side = int(rng.integers(obs_sides[0], obs_sides[1] + 1))
        reqs.append(Request(i, int(rng.integers(0, n_problems)), side, float(rng.uniform(0.05, 0.95)),
                            float(arrivals[i])))
    return reqs


def measure(n_problems: int = 64, n_requests: int = 10000, loads=(0.5, 0.8, 1.0), sides=(16, 64),
            H_range=(64, 256), obs_sides=(8, 48), seed: int = 11, tick_s: float = 0.02,
            n_streams: int = 4, max_batch: int = 32, memory_budget: Optional[float] = None,
            n_samples: int = 0):
    """Latency of Poisson-arriving requests against resident problems.

    First the saturated throughput (every request arrives at once), then, for
    each load factor f, a fresh stream of requests arriving at f times that
    rate; one slice is pushed to every problem per tick throughout.  Returns the
    percentiles per load and the resident memory.  The device-memory budget
    (resident histories, cached views and outputs) defaults to 64 GB.

    With n_samples > 0 the outputs of that many seeded requests of the last
    load level are kept and (result, samples) is returned; each sample holds
    what an independent check needs to recompute the request (see
    ``served_sample``)."""
    import torch

    if memory_budget is None:
        memory_budget = 64e9
    probs = make_problems(n_problems, seed, sides=sides, H_range=H_range)
    # saturated throughput under the same slice pushes as the load levels
    # (every request arrives at once; the pushes compete for the device and
    # the host loop, so a rate measured without them overstates capacity)
    eng = ServingEngine(probs, obs_half_width=2.0, n_streams=n_streams, max_batch=max_batch, tick_s=tick_s,
                        memory_budget=memory_budget)
    sat = eng.run(poisson_requests(n_requests, rate=1e9, n_problems=n_problems, obs_sides=obs_sides,
                                   seed=seed + 1))
    out = {"problems": n_problems, "requests_per_load": n_requests, "source_sides": list(sides),
           "memory_budget_bytes": int(memory_budget),
           "history_slices": list(H_range), "obs_sides": list(obs_sides),
           "resident_ring_bytes": int(eng.resident_bytes),
           "saturated": {"requests_per_s": sat.requests_per_s, "pairs_per_s": sat.pairs_per_s,
                         "mean_batch": sat.mean_batch}, "loads": []}
    samples = []
    for i, f in enumerate(loads):
        rate = f * sat.requests_per_s
        reqs = poisson_requests(n_requests, rate=rate, n_problems=n_problems, obs_sides=obs_sides,
                                seed=seed + 2 + i)
        if n_samples and i == len(loads) - 1:
            pick = np.random.Generator(np.random.PCG64(seed + 99)).choice(len(reqs), n_samples, replace=False)
            eng.keep_ids = {int(k) for k in pick}
        st = eng.run(reqs)
        out["loads"].append({"load": f, "offered_requests_per_s": rate, "p50_ms": st.p50_ms,
                             "p99_ms": st.p99_ms, "mean_ms": st.mean_ms,
                             "requests_per_s": st.requests_per_s, "pairs_per_s": st.pairs_per_s,
                             "completed": st.completed, "rejected": st.rejected, "evicted": st.evicted,
                             "failed": st.failed, "mean_batch": st.mean_batch,
                             "peak_device_bytes": st.peak_bytes})
        if eng.keep_ids:
            samples = [served_sample(eng, r) for r in reqs if r.rid in eng.keep_ids and r.E is not None
                       and not r.error]
            eng.keep_ids = set()
    eng.close()
    torch.cuda.synchronize()
    return (out, samples) if n_samples else out


def served_sample(eng: "ServingEngine", req: Request) -> dict:
    """What an independent check needs to recompute one served request: the
    problem's source grid, source model and dt (slice n is the model at n dt,
    t0 = 0), the observation grid, the time, and the result copied to the host."""
    p = eng.problems[req.problem]
    s = req.obs_side
    L = eng.obs_half_width
    return {"rid": req.rid, "src_side": p.side, "src_half_width": p.L, "dt": p.dt, "model": p.model,
            "obs_side": s, "obs_half_width": L, "t": req.t, "n_pushed": p.n_pushed,
            "E": req.E.cpu().numpy(), "B": req.B.cpu().numpy()}


def measure_batch(n_problems: int = 256, sides=(8, 48), H_range=(32, 128), obs_sides=(8, 32), seed: int = 4,
                  reps: int = 3) -> dict:
    """Independent problems of uneven sizes in one batched evaluation: source
    grids of side uniform in `sides`, histories uniform in H_range, one
    observation grid per problem of side uniform in obs_sides (over a box
    twice the source box) at one time inside its window; every problem's
    result comes out of one jefi_eval_batch call (one persistent launch per
    kernel variant, then one reduction).  Returns the time of the call and
    the pair rate; then the same batch as a batch plan (one CUDA-graph
    launch per call), before and after the plan's autotuner."""
    import torch

    probs = make_problems(n_problems, seed, sides=sides, H_range=H_range)
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    views, ts, Es, Bs, pairs = [], [], [], [], 0
    for p in probs:
        s = int(rng.integers(obs_sides[0], obs_sides[1] + 1))
        g = grid((s,) * 3, (-2.0,) * 3, (4.0 / s,) * 3)
        v = jefi_create_view(p.handle, obs_grid=g)
        lo, hi = jefi_valid_window(v)
        if not math.isfinite(lo):
            lo = hi - 4 * p.dt
        views.append(v)
        ts.append(lo + (hi - lo) * float(rng.uniform(0.05, 0.95)))
        Es.append(torch.empty((s ** 3, 3), dtype=torch.float64, device="cuda"))
        Bs.append(torch.empty_like(Es[-1]))
        pairs += p.side ** 3 * s ** 3
    jefi_eval_batch(views, ts, Es, Bs)                 # warm-up
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        jefi_eval_batch(views, ts, Es, Bs)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    bands = [jefi_get_info(v)["staged_band"] for v in views]
    out = {"problems": n_problems, "source_sides": list(sides), "history_slices": list(H_range),
           "obs_sides": list(obs_sides), "pairs": pairs, "ms_per_batch": ms, "pairs_per_s": pairs / (ms / 1e3),
           "staged_problems": sum(1 for b in bands if b > 0)}

    # Each kernel variant's problems as a batch of their own: where the
    # batch's time goes (the staged band of each view, 0 = direct gather).
    by_kernel = {}
    try:
        groups = {}
        for i, b in enumerate(bands):
            groups.setdefault(int(b), []).append(i)
        for b, idx in sorted(groups.items()):
            sub = ([views[i] for i in idx], [ts[i] for i in idx], [Es[i] for i in idx], [Bs[i] for i in idx])
            jefi_eval_batch(*sub)                     # warm-up
            torch.cuda.synchronize()
            e0.record()
            jefi_eval_batch(*sub)
            e1.record()
            torch.cuda.synchronize()
            ms_b = e0.elapsed_time(e1)
            pairs_b = sum(probs[i].side ** 3 * Es[i].shape[0] for i in idx)
            by_kernel[str(b)] = {"problems": len(idx), "pairs": pairs_b, "ms": ms_b,
                                 "pairs_per_s": pairs_b / (ms_b / 1e3)}
        out["by_kernel"] = by_kernel
    except Exception as e:      # a diagnostic: never lose the batch measurement to it
        out["by_kernel_error"] = f"{type(e).__name__}: {e}"

    def time_plan(plan):
        jefi_batch_plan_launch(plan, ts)              # warm-up
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            jefi_batch_plan_launch(plan, ts)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    plan = None
    try:
        plan = jefi_batch_plan_create(views, Es, Bs)
        ms_graph = time_plan(plan)
        out["graph"] = {"ms_per_batch": ms_graph, "pairs_per_s": pairs / (ms_graph / 1e3)}
        rep = jefi_batch_plan_tune(plan, ts)
        ms_tuned = time_plan(plan)
        bands = [jefi_get_info(v)["staged_band"] for v in views]
        out["tuned"] = {"ms_per_batch": ms_tuned, "pairs_per_s": pairs / (ms_tuned / 1e3),
                        "staged_problems": sum(1 for b in bands if b > 0), "tuner": rep}
    except JefiError as e:
        out["plan_error"] = str(e)
    finally:
        if plan is not None:
            jefi_batch_plan_destroy(plan)
    out["device_status"] = max(jefi_get_info(v)["device_status"] for v in views)
    for v in views:
        jefi_destroy(v)
    for p in probs:
        jefi_destroy(p.handle)
    return out


def measure_single(src_side: int, obs_side: int, H: int, reps: int = 3, seed: int = 9) -> dict:
    """One resident problem of the serving kind (source grid over [-1,1]^3,
    observation grid over [-2,2]^3 as a view, dt = R_max/(c (H-8))) and the
    time of one evaluation in its valid window."""
    import torch

    rmax = math.sqrt(3.0) * 3.0
    dt = rmax / (H - 8)
    rng = np.random.Generator(np.random.PCG64(seed))
    blobs = [OscBlob(float(q), (float(rng.uniform(0.2, 0.3)),) * 3, tuple(rng.uniform(-0.2, 0.2, 3)),
                     tuple(rng.uniform(-0.3, 0.3, 3)), 1.0) for q in (1.0, -1.0)]
    p = ServedProblem(src_side, 1.0, H, dt, blobs)
    s = torch.cuda.current_stream()
    for _ in range(H + 1):
        p.push_next(s)
    g = grid((obs_side,) * 3, (-2.0,) * 3, (4.0 / obs_side,) * 3)
    v = jefi_create_view(p.handle, obs_grid=g)
    lo, hi = jefi_valid_window(v)
    t = 0.5 * (lo + hi) if math.isfinite(lo) else hi - 2 * dt
    E = torch.empty((obs_side ** 3, 3), dtype=torch.float64, device="cuda")
    B = torch.empty_like(E)
    from . import jefi_eval_fields

    jefi_eval_fields(v, t, E, B)                       # warm-up
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        jefi_eval_fields(v, t, E, B)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    info = jefi_get_info(v)
    pairs = src_side ** 3 * obs_side ** 3
    out = {"source_side": src_side, "obs_side": obs_side, "history_slices": H, "dt": dt, "ms": ms,
           "pairs_per_s": pairs / (ms / 1e3), "staged_band": info["staged_band"], "n_split": info["n_split"],
           "slot_fallbacks": info["slot_fallbacks"], "device_status": info["device_status"]}
    jefi_destroy(v)
    jefi_destroy(p.handle)
    return out


def main(argv=None):
    import argparse
    import json

    ap = argparse.ArgumentParser(description="Serving latency of jefi field requests (p50/p99 per load).")
    ap.add_argument("--problems", type=int, default=64)
    ap.add_argument("--requests", type=int, default=10000, help="requests per load level")
    ap.add_argument("--loads", default="0.5,0.8,1.0", help="fractions of the saturated request rate")
    ap.add_argument("--sides", default="16,64", help="source grid side range")
    ap.add_argument("--history", default="64,256", help="resident history length range")
    ap.add_argument("--obs-sides", default="8,48", help="observation grid side range")
    ap.add_argument("--seed", type=int, default=11)
    ap.add_argument("--tick-ms", type=float, default=20.0, help="one slice pushed per problem per tick")
    ap.add_argument("--budget-gb", type=float, default=None,
                    help="device memory for histories, views and outputs (default: 64 GB)")
    ap.add_argument("--single", default=None, metavar="SRC,OBS,H",
                    help="time one evaluation of one problem (source side, observation side, history)")
    ap.add_argument("--reps", type=int, default=3, help="evaluations timed with --single")
    a = ap.parse_args(argv)
    pair = lambda s: tuple(int(x) for x in s.split(","))
    if a.single:
        src_side, obs_side, H = pair(a.single)
        print(json.dumps(measure_single(src_side, obs_side, H, a.reps)))
        return
    res = measure(a.problems, a.requests, tuple(float(x) for x in a.loads.split(",")), pair(a.sides),
                  pair(a.history), pair(a.obs_sides), a.seed, a.tick_ms / 1e3,
                  memory_budget=None if a.budget_gb is None else a.budget_gb * 1e9)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
