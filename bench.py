#!/usr/bin/env python3
"""Benchmark: Jefimenko retarded direct sum on GB300 (pair-interactions per second).

Workload (one "step" = one pass of the whole hot path): the heavy-ion-shaped
problem -- source and observation grids both 64^3 over [-5,5]^3, two
Lorentz-contracted Gaussian charges at +-0.995c with 1% seeded noise, a
128-slice resident history -- push one new source slice, then evaluate E and
B at 8 times spread over the valid window (one launch).  Pairs per step =
64^3 * 64^3 * 8 = 5.5e11.  The ring (1.08 GB FP32) is larger than L2, so no
flush is needed between steps.

Output: one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on a bounded sample (the paper is the only artifact: there is
no reference code to run).
Multi-GPU runs (torchrun) are independent replicas: the path needs no
exchange, so each rank runs the full workload on its own GPU ("weak").
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair-interactions/s, compensated FP32 vs plain FP64 at 1e-5 err; serving p50/p99"
UNIT = "pairs/s"
# Canonical FP32 pipe instructions per pair: D (3 FADD), S (1 FMUL + 2 FFMA), R (1 FMUL),
# slot (1 FFMA + 1 floor), r^-2 and r^-3 (2 FMUL), the scalar E term (1 FMUL + 1 FFMA),
# E (6 FFMA), V (3 FMUL + 3 FFMA), B (6 FFMA): 3 FADD + 8 FMUL + 19 FFMA + 1 floor = 31.
SUM_FP32_INSTR_PER_PAIR = 31
# The same algorithm in FP64 (the plain FP64 path): the 31 operations above as
# DADD/DMUL/DFMA; the FP64 reciprocal square root's Newton steps and the
# threshold compares are not counted as useful work.
SUM_FP64_INSTR_PER_PAIR = 31
FP32_LANES_PER_SM = 128
# FP64 FMA results per SM per clock on GB300: 2.  An FMA throughput probe
# (1216 CTAs x 256 threads x 8 independent DFMA chains) measured 1.994 DFMA
# per SM per clock at 2070 MHz (FFMA: 124.7 of 128); the part's nominal
# 1.25 TFLOP/s FP64 is the same figure (152 x 2 x 2 FLOP x 2.07 GHz).
FP64_LANES_PER_SM = 2
DEFAULT_SM_MAX_MHZ = 2070.0


def device_sm_count(dev) -> int:
    """Streaming multiprocessors of the device (the roofline's unit count)."""
    import torch

    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def sm_max_mhz(clk) -> float:
    """Maximum SM clock: from the nvidia-smi samples, else the part's 2070 MHz."""
    if clk and clk.get("sm_max_mhz"):
        return float(clk["sm_max_mhz"])
    return DEFAULT_SM_MAX_MHZ


def pipe_peak(n_sm: int, lanes: int, mhz: float) -> float:
    """Instructions per second of one arithmetic pipe over the whole GPU."""
    return n_sm * lanes * mhz * 1e6


# ---------------------------------------------------------------------------- distributed
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_dist(world, backend):
    import torch.distributed as dist

    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return dist


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest value of x over all ranks (the job is as slow as its slowest rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200",
                                          "-i", str(self.gpu)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r)
                          if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": rows[0][1],
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------- workload
def eval_times(lo, hi, k=8):
    return [lo + (hi - lo) * (i + 0.5) / k for i in range(k)]


def kernel_source_hash():
    """Hash of the sources of the dominant kernel (the staged FP32 sum)."""
    h = hashlib.sha256()
    for f in ("jefi_staged.cuh", "jefi_staged.cu", "jefi_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2104_05426_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per sum-kernel launch from the committed ncu summary, if it
    was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "sum_f32c_c2_ncu.md")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256") != kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_full_launch"])
    except (KeyError, ValueError):
        return None


def run_gpu(args):
    import torch

    import paper_2104_05426_gb300 as jefi
    from workloads import c2_heavy_ion

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = init_dist(world, "nccl")
    stream = torch.cuda.current_stream()

    p = c2_heavy_ion(side=args.side)
    H = p.H
    n_extra = args.warmup + 2 * args.steps
    slices = [p.source.sample(p.src, p.t0 + n * p.dt, n) for n in range(H + n_extra)]
    dev_slices = [(torch.from_numpy(r).to(dev), torch.from_numpy(j).to(dev)) for r, j in slices]

    def make(prec, flags=0, first_slice=0):
        # a handle whose slice 0 is workload slice `first_slice`
        prm = jefi.default_params(c=p.c, k_e=p.k_e, k_b=p.k_b, dt=p.dt,
                                  t0=p.t0 + first_slice * p.dt, history_slots=H,
                                  precision=prec, flags=flags)
        return jefi.jefi_create(jefi.grid_from(p.src), obs_grid=jefi.grid_from(p.obs_grid),
                                params=prm, torch_allocator=True)

    h = make(args.precision, jefi.JEFI_FLAG_STATS)
    for n in range(H):
        jefi.jefi_push_sources(h, *dev_slices[n])
    n_obs = p.n_obs
    n_src = p.src.size
    n_t = 8
    pairs_step = n_obs * n_src * n_t
    E = torch.empty((n_t, n_obs, 3), dtype=torch.float64, device=dev)
    B = torch.empty_like(E)

    # Evaluation times: the workload's 8 interior times of the initial window,
    # slid by dt per pushed slice (the window moves by exactly one slice).
    def times_now(n_latest):
        return [t + (n_latest - (H - 1)) * p.dt for t in p.times]

    # first evaluation (untimed): accuracy reference for the oracle sample
    t_first = times_now(H - 1)
    jefi.jefi_eval_fields_multi(h, t_first, E, B)
    E_first, B_first = E.cpu().numpy(), B.cpu().numpy()

    next_slice = H

    def step(host_io=False, E_host=None, B_host=None, pinned=None):
        nonlocal next_slice
        if host_io:
            jefi.jefi_push_sources(h, pinned[next_slice][0], pinned[next_slice][1])
        else:
            jefi.jefi_push_sources(h, *dev_slices[next_slice])
        next_slice += 1
        ts = times_now(next_slice - 1)
        if host_io:
            jefi.jefi_eval_fields_multi(h, ts, E_host, B_host)
        else:
            jefi.jefi_eval_fields_multi(h, ts, E, B)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    jefi.jefi_reset_stats(h)
    launches0 = jefi.jefi_get_info(h)["kernel_launches"]
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    ms_local = ev0.elapsed_time(ev1)
    info = jefi.jefi_get_info(h)
    launches = info["kernel_launches"] - launches0
    ms = max_over_ranks(ms_local, world, dev)
    value = world * pairs_step * args.steps / (ms / 1e3)

    # dominant kernel: the sum kernel, timed by the library's events on this stream
    sum_ms = info["sum_ms_total"] / max(info["sum_launches"], 1)
    pairs_launch = pairs_step
    n_sm = device_sm_count(dev)
    mhz = sm_max_mhz(clk)
    if args.precision == "fp64":
        instr, lanes, unit, kname = SUM_FP64_INSTR_PER_PAIR, FP64_LANES_PER_SM, "FP64 Tinstr/s", "sum_f64_kernel"
    else:
        instr, lanes, unit = SUM_FP32_INSTR_PER_PAIR, FP32_LANES_PER_SM, "FP32 Tinstr/s"
        kname = (f"sum_f32_staged_kernel<band={info['staged_band']}>" if info["staged_band"]
                 else "sum_f32_kernel (direct gather)")
    achieved = pairs_launch * instr / (sum_ms / 1e3) / 1e12
    peak = pipe_peak(n_sm, lanes, mhz) / 1e12
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3),
                "unit": unit, "frac": round(achieved / peak, 4),
                "traffic": profiled_traffic() if args.precision == "fp32c" and args.side == 64 else None,
                "kernel": kname, "device_status": info["device_status"],
                "kernel_ms": round(sum_ms, 3), "fallback_pairs": info["slot_fallbacks"],
                "peak_basis": f"{n_sm} SMs (device query) x {lanes} {unit.split()[0]} lanes x "
                              f"{mhz:.0f} MHz (max SM clock); {instr} instructions per pair"}

    # end to end through the C ABI with pinned host buffers
    pinned = [(torch.from_numpy(r).pin_memory(), torch.from_numpy(j).pin_memory())
              for r, j in slices]
    E_host = torch.empty((n_t, n_obs, 3), dtype=torch.float64).pin_memory()
    B_host = torch.empty_like(E_host).pin_memory()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(True, E_host, B_host, pinned)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e = {"value": world * pairs_step * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": n_src * 4 * 8, "d2h_bytes_per_step": 2 * n_t * n_obs * 3 * 8}

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
              "config": {"workload": f"heavy-ion {args.side}^3 src x {args.side}^3 obs over [-5,5]^3, "
                                     "2 Gaussian charges +-0.995c + 1% noise, H=128, 8 eval times "
                                     "per step",
                         "precision": {"fp32c": "fp32 compensated, fp64 cross-split reduction",
                                       "fp32": "fp32, fp64 cross-split reduction",
                                       "fp64": "fp64"}[args.precision],
                         "pairs_per_step": pairs_step, "l2": "inputs larger than L2 (FP32 ring "
                         f"{n_src * (H + info['staged_band'] + 1) * 32 / 1e9:.2f} GB)",
                         "parallelism": f"replicas x{world}"},
              "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk}

    if rank == 0 and not args.no_extras:
        # plain FP64 GPU path on the same workload (one evaluation time)
        h64 = make("fp64", jefi.JEFI_FLAG_STATS, first_slice=next_slice - H)
        for n in range(next_slice - H, next_slice):
            jefi.jefi_push_sources(h64, *dev_slices[n])
        tmid = times_now(next_slice - 1)[n_t // 2]
        E64 = torch.empty((1, n_obs, 3), dtype=torch.float64, device=dev)
        B64 = torch.empty_like(E64)
        jefi.jefi_eval_fields_multi(h64, [tmid], E64, B64)      # warm-up
        jefi.jefi_reset_stats(h64)
        jefi.jefi_eval_fields_multi(h64, [tmid], E64, B64)
        i64 = jefi.jefi_get_info(h64)
        ms64 = i64["sum_ms_total"] / max(i64["sum_launches"], 1)
        jefi.jefi_eval_fields_multi(h, [tmid], E[:1], B[:1])
        torch.cuda.synchronize()
        err = {"E": float(torch.linalg.norm(E[0] - E64[0]) / torch.linalg.norm(E64[0])),
               "B": float(torch.linalg.norm(B[0] - B64[0]) / torch.linalg.norm(B64[0]))}
        fp32c_kernel_pairs_s = pairs_launch / (sum_ms / 1e3)
        fp64_pairs_s = n_obs * n_src / (ms64 / 1e3)
        fp64_peak = pipe_peak(n_sm, FP64_LANES_PER_SM, mhz)
        fp64_ach = fp64_pairs_s * SUM_FP64_INSTR_PER_PAIR
        result["fp64_plain"] = {"value": fp64_pairs_s, "unit": UNIT, "kernel_ms": ms64,
                                "fp32c_speedup_kernel": fp32c_kernel_pairs_s / fp64_pairs_s,
                                "rel_l2_fp32c_vs_fp64_all_points": err,
                                "roofline": {"bound": "alu", "achieved": round(fp64_ach / 1e12, 4),
                                             "peak": round(fp64_peak / 1e12, 4), "unit": "FP64 Tinstr/s",
                                             "frac": round(fp64_ach / fp64_peak, 4),
                                             "peak_basis": f"{n_sm} SMs x {FP64_LANES_PER_SM} FP64 lanes (DFMA "
                                                           f"probe: 1.994 per SM per clock) x {mhz:.0f} MHz; "
                                                           f"{SUM_FP64_INSTR_PER_PAIR} instructions per pair"}}
        # plain FP32 (no compensation) on the same 8-time launch: what the
        # compensation costs, and what it buys against the FP64 path
        h32 = make("fp32", jefi.JEFI_FLAG_STATS, first_slice=next_slice - H)
        for n in range(next_slice - H, next_slice):
            jefi.jefi_push_sources(h32, *dev_slices[n])
        ts_now = times_now(next_slice - 1)
        jefi.jefi_eval_fields_multi(h32, ts_now, E, B)         # warm-up
        jefi.jefi_reset_stats(h32)
        for _ in range(3):
            jefi.jefi_eval_fields_multi(h32, ts_now, E, B)
        i32 = jefi.jefi_get_info(h32)
        ms32 = i32["sum_ms_total"] / max(i32["sum_launches"], 1)
        jefi.jefi_eval_fields_multi(h32, [tmid], E[:1], B[:1])
        torch.cuda.synchronize()
        err32 = {"E": float(torch.linalg.norm(E[0] - E64[0]) / torch.linalg.norm(E64[0])),
                 "B": float(torch.linalg.norm(B[0] - B64[0]) / torch.linalg.norm(B64[0]))}
        result["fp32_plain"] = {"value": pairs_launch / (ms32 / 1e3), "unit": UNIT, "kernel_ms": ms32,
                                "compensation_cost": sum_ms / ms32 - 1.0,
                                "rel_l2_fp32_vs_fp64_all_points": err32,
                                "rel_l2_fp32c_vs_fp64_all_points": err,
                                "note": "same 8-time launch without the Kahan step per brick"}
        jefi.jefi_destroy(h32)
        jefi.jefi_destroy(h64)
        result["so_decomposition"] = so_leg(p, dev_slices, next_slice, H, times_now(next_slice - 1)[n_t // 2],
                                            E64[0], B64[0])
        # second-order retarded time (opt-in) on the same workload, 8 times per
        # launch: central differences read two slices past the slot, so the
        # handle holds two more slices and the times sit two slices back
        prm_i = jefi.default_params(c=p.c, k_e=p.k_e, k_b=p.k_b, dt=p.dt,
                                    t0=p.t0 + (next_slice - H - 2) * p.dt, history_slots=H + 2,
                                    precision="fp32c", flags=jefi.JEFI_FLAG_STATS | jefi.JEFI_FLAG_INTERP)
        hi2 = jefi.jefi_create(jefi.grid_from(p.src), obs_grid=jefi.grid_from(p.obs_grid), params=prm_i,
                               torch_allocator=True)
        for n in range(next_slice - H - 2, next_slice):
            jefi.jefi_push_sources(hi2, *dev_slices[n])
        ts_i = times_now(next_slice - 3)
        jefi.jefi_eval_fields_multi(hi2, ts_i, E, B)      # warm-up
        jefi.jefi_reset_stats(hi2)
        jefi.jefi_eval_fields_multi(hi2, ts_i, E, B)
        ii = jefi.jefi_get_info(hi2)
        ms_i = ii["sum_ms_total"] / max(ii["sum_launches"], 1)
        result["interp_fp32c"] = {"value": pairs_launch / (ms_i / 1e3), "unit": UNIT, "kernel_ms": ms_i,
                                  "vs_floor_rule_kernel": sum_ms / ms_i,
                                  "device_status": ii["device_status"],
                                  "note": "JEFI_FLAG_INTERP: sources interpolated at the retarded "
                                          "time, central differences; same 8-time launch"}
        jefi.jefi_destroy(hi2)
        result["dipole"] = dipole_leg(dev)
        if not args.no_serving:
            result["serving"], served = serving_leg()
            from paper_2104_05426_gb300.serving import measure_batch

            result["batch"] = dict(measure_batch(),
                                   workload="256 independent problems (source sides 8-48, histories "
                                            "32-128, observation sides 8-32) in one jefi_eval_batch call; "
                                            "graph: the same batch as a batch plan (one CUDA-graph launch); "
                                            "tuned: after the plan's autotuner (kernels, source splits)")
        if not args.no_cpu_baseline:
            result["cpu_baseline"], result["oracle_check"] = cpu_baseline(p, slices[:H], t_first,
                                                                          E_first, B_first)
            if not args.no_serving:
                try:
                    result["serving"]["oracle_check"] = served_oracle_check(served, point_stride=31)
                except Exception as e:      # a diagnostic: never lose the benchmark line to it
                    result["serving"]["oracle_check_error"] = f"{type(e).__name__}: {e}"
            try:
                result["oracle_check"]["configs"] = config_errors(dev)
            except Exception as e:      # a diagnostic: never lose the benchmark line to it
                result["oracle_check"]["configs_error"] = f"{type(e).__name__}: {e}"
    jefi.jefi_destroy(h)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.destroy_process_group()


def so_leg(p, dev_slices, next_slice, H, t, E64, B64, parts=(2, 1, 1), reps=3):
    """The paper's S-O decomposition (Sec. 2.2, Fig. 2) of the heavy-ion
    workload on this one GPU: the source grid in `parts` brick-aligned boxes,
    one handle per (box, all observation points) pair fed from the whole
    grid's slices, the fields summed in box order by jefi_sum_fields.  Its
    evaluation time against the whole problem's, and its FP64 fields against
    the whole FP64 handle's."""
    import torch

    import paper_2104_05426_gb300 as jefi
    from paper_2104_05426_gb300.decomp import SODecomposition

    g = jefi.grid_from(p.src)
    prm = dict(c=p.c, k_e=p.k_e, k_b=p.k_b, dt=p.dt, t0=p.t0 + (next_slice - H) * p.dt, history_slots=H)
    out = {"parts": list(parts), "workload": "heavy-ion source grid in brick-aligned boxes, all observers"}
    for prec in ("fp32c", "fp64"):
        so = SODecomposition(g, p.obs_grid.points(), dict(prm, precision=prec, flags=jefi.JEFI_FLAG_STATS),
                             src_parts=parts, torch_allocator=True)
        for n in range(next_slice - H, next_slice):
            so.push(*dev_slices[n])
        n_rep = reps if prec == "fp32c" else 1           # FP64: one evaluation (its accuracy only)
        if prec == "fp32c":
            so.fields(t)                                 # warm-up
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(n_rep):
            E, B = so.fields(t)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n_rep
        out[prec] = {"ms_per_eval": ms, "pairs_per_s": p.n_obs * p.src.size / (ms / 1e3),
                     "rel_l2_vs_whole_fp64": {
                         "E": float(torch.linalg.norm(E - E64) / torch.linalg.norm(E64)),
                         "B": float(torch.linalg.norm(B - B64) / torch.linalg.norm(B64))}}
        so.close()
    return out


def dipole_leg(dev, reps=5):
    """The oscillating-dipole workload (32^3 sources over [-0.5,0.5]^3, 4096
    points on shells R = 5, 10, 20, 40, 256-slice history, backward
    differences): 4 evaluation times per launch, compensated FP32 and FP64.
    Reports pairs/s from the library's kernel events, the FP32 pipe fraction
    of the compensated path (same canonical count as the benchmark) and its
    rel-L2 against the FP64 GPU path per shell (the FP64 path matches the
    oracle to 1e-12 in the test suite)."""
    import torch

    import paper_2104_05426_gb300 as jefi
    from workloads import c3_dipole

    p = c3_dipole()
    rho, J, _, _ = p.source.history(p.src, p.n_push, p.dt, p.t0)
    slices = [(torch.from_numpy(np.ascontiguousarray(rho[n])).to(dev),
               torch.from_numpy(np.ascontiguousarray(J[n])).to(dev)) for n in range(p.n_push)]
    n_obs, n_src, n_t = len(p.obs_points), p.src.size, len(p.times)
    pairs = n_obs * n_src * n_t
    out, fields = {}, {}
    for prec in ("fp32c", "fp64"):
        prm = jefi.default_params(c=p.c, k_e=p.k_e, k_b=p.k_b, dt=p.dt, t0=p.t0, history_slots=p.H,
                                  precision=prec, flags=jefi.JEFI_FLAG_STATS)
        h = jefi.jefi_create(jefi.grid_from(p.src), obs_points=p.obs_points, params=prm,
                             torch_allocator=True)
        for r_n, j_n in slices:
            jefi.jefi_push_sources(h, r_n, j_n)
        E = torch.empty((n_t, n_obs, 3), dtype=torch.float64, device=dev)
        B = torch.empty_like(E)
        jefi.jefi_eval_fields_multi(h, p.times, E, B)          # warm-up
        jefi.jefi_reset_stats(h)
        for _ in range(reps if prec == "fp32c" else 1):
            jefi.jefi_eval_fields_multi(h, p.times, E, B)
        info = jefi.jefi_get_info(h)
        ms = info["sum_ms_total"] / max(info["sum_launches"], 1)
        out[prec] = {"value": pairs / (ms / 1e3), "unit": UNIT, "kernel_ms": ms,
                     "kernel": (f"staged band {info['staged_band']}" if info["staged_band"] and prec != "fp64"
                                else ("sum_f64_kernel" if prec == "fp64" else "sum_f32_kernel (direct gather)")),
                     "device_status": info["device_status"],
                     "fallback_pairs_per_launch": info["slot_fallbacks"] / max(info["sum_launches"], 1)}
        fields[prec] = (E, B)
        jefi.jefi_destroy(h)
    peak = pipe_peak(device_sm_count(dev), FP32_LANES_PER_SM, DEFAULT_SM_MAX_MHZ)
    out["fp32c"]["fp32_pipe_frac"] = out["fp32c"]["value"] * SUM_FP32_INSTR_PER_PAIR / peak
    out["fp32c_speedup_kernel"] = out["fp32c"]["value"] / out["fp64"]["value"]
    radii = np.linalg.norm(p.obs_points, axis=1)
    errs = {}
    for R in (5.0, 10.0, 20.0, 40.0):
        m = torch.from_numpy(np.abs(radii - R) < 1e-6 * R).to(dev)
        errs[str(R)] = max(float(torch.linalg.norm(fields["fp32c"][k][:, m] - fields["fp64"][k][:, m]) /
                                 torch.linalg.norm(fields["fp64"][k][:, m])) for k in (0, 1))
    out["rel_l2_fp32c_vs_fp64_by_shell"] = errs
    out["workload"] = ("oscillating dipole: 32^3 sources over [-0.5,0.5]^3, 4096 points on shells "
                       "R = 5, 10, 20, 40, H = 256, 4 times per launch, backward differences")
    out["pairs_per_launch"] = pairs
    return out


def serving_leg(n_problems=16, n_requests=600, seed=11, tick_s=0.02, n_samples=6):
    """Continuous batching of Poisson-arriving requests against resident
    problems (source sides 16-48, histories 64-128 slices, observation sides
    8-48, one slice pushed to every problem per tick): saturated throughput
    first (all requests at once, pushes running), then p50/p99 latency at
    0.8x that rate.
    Returns the figures and a seeded sample of served requests (kept for the
    oracle check)."""
    from paper_2104_05426_gb300.serving import ServingEngine, make_problems, poisson_requests, served_sample

    probs = make_problems(n_problems, seed, sides=(16, 48), H_range=(64, 128))
    sides = [8, 16, 24, 32, 40, 48]
    # saturated under the same pushes as the measured load
    eng = ServingEngine(probs, obs_half_width=2.0, n_streams=4, max_batch=32, tick_s=tick_s)
    sat = eng.run(poisson_requests(n_requests, rate=1e9, n_problems=n_problems, seed=seed + 1,
                                   side_choices=sides))
    rate = 0.8 * sat.requests_per_s
    reqs = poisson_requests(n_requests, rate=rate, n_problems=n_problems, seed=seed + 2, side_choices=sides)
    eng.keep_ids = {int(k) for k in np.random.Generator(np.random.PCG64(seed + 3)).choice(
        n_requests, n_samples, replace=False)}
    st = eng.run(reqs)
    samples = [served_sample(eng, r) for r in reqs if r.rid in eng.keep_ids and not r.error]
    eng.close()
    return {"p50_ms": st.p50_ms, "p99_ms": st.p99_ms, "mean_ms": st.mean_ms,
            "offered_requests_per_s": rate, "requests_per_s": st.requests_per_s,
            "pairs_per_s": st.pairs_per_s, "saturated_requests_per_s": sat.requests_per_s,
            "saturated_pairs_per_s": sat.pairs_per_s, "completed": st.completed,
            "rejected": st.rejected, "evicted": st.evicted, "failed": st.failed,
            "mean_batch": st.mean_batch, "max_batch": st.max_batch,
            "peak_device_bytes": st.peak_bytes,
            "workload": f"{n_problems} resident problems, {n_requests} Poisson requests at 0.8x "
                        f"saturation, obs sides {sides}, slice push every {tick_s * 1e3:.0f} ms, "
                        "compensated FP32"}, samples


def served_oracle_check(samples, point_stride=1):
    """Served requests recomputed by the FP64 CPU oracle from the same source
    model (slice n at n dt), on every point_stride-th observation point:
    rel-L2 per field, worst over the sample."""
    import oracle
    from workloads import Grid

    worst = {"E": 0.0, "B": 0.0}
    pairs = 0
    t_start = time.perf_counter()
    for sm in samples:
        src = Grid.cube(sm["src_side"], -sm["src_half_width"], sm["src_half_width"])
        obs_all = Grid.cube(sm["obs_side"], -sm["obs_half_width"], sm["obs_half_width"]).points()
        idx = np.arange(0, len(obs_all), point_stride)
        dt, t = sm["dt"], sm["t"]
        model = sm["model"]
        rmax = math.sqrt(3.0) * (sm["src_half_width"] + sm["obs_half_width"])
        n_lo = max(0, int(math.floor((t - rmax) / dt)) - 2)
        n_hi = min(sm["n_pushed"] - 1, int(math.ceil(t / dt)) + 1)
        hist = [model.sample(src, n * dt) for n in range(n_lo, n_hi + 1)]
        rho = np.stack([h[0] for h in hist])
        J = np.stack([h[1] for h in hist])
        Er, Br = oracle.fields(src.n, src.lo, src.d, obs_all[idx], rho, J, dt=dt, t0=n_lo * dt, t=t)
        for k, got, ref in (("E", sm["E"][idx], Er), ("B", sm["B"][idx], Br)):
            worst[k] = max(worst[k], float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
        pairs += len(idx) * src.size
    return {"requests": len(samples), "point_stride": point_stride, "pairs": pairs,
            "rel_l2_worst": worst, "seconds": time.perf_counter() - t_start}


def cpu_baseline(p, slices, times, E_gpu, B_gpu, stride=512):
    """FP64 oracle on every `stride`-th observation point, all sources, all 8
    times (about 1.1e9 pairs), on every host core; also checks the GPU result
    on that sample."""
    import oracle

    rho = np.stack([s[0] for s in slices])
    J = np.stack([s[1] for s in slices])
    sub = np.arange(0, p.n_obs, stride)
    obs = p.obs()[sub]
    cores = oracle.max_threads()
    t0 = time.perf_counter()
    errs = {"E": 0.0, "B": 0.0}
    for i, t in enumerate(times):
        Er, Br = oracle.fields(p.src.n, p.src.lo, p.src.d, obs, rho, J, dt=p.dt, t0=p.t0, t=t)
        errs["E"] = max(errs["E"], float(np.linalg.norm(E_gpu[i][sub] - Er) / np.linalg.norm(Er)))
        errs["B"] = max(errs["B"], float(np.linalg.norm(B_gpu[i][sub] - Br) / np.linalg.norm(Br)))
    dt_s = time.perf_counter() - t0
    pairs = len(sub) * p.src.size * len(times)
    # one core, for comparison with single-threaded figures
    sub1 = np.arange(0, p.n_obs, 16 * stride)
    t1 = time.perf_counter()
    oracle.fields(p.src.n, p.src.lo, p.src.d, p.obs()[sub1], rho, J, dt=p.dt, t0=p.t0, t=times[0],
                  threads=1)
    dt1 = time.perf_counter() - t1
    base = {"value": pairs / dt_s, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"every {stride}th of {p.n_obs} observation points x {p.src.size} sources x "
                      f"{len(times)} times = {pairs:.3e} pairs, {dt_s:.1f} s",
            "single_core_value": len(sub1) * p.src.size / dt1,
            "single_core_sample": f"every {16 * stride}th observation point x {p.src.size} sources x "
                                  f"1 time = {len(sub1) * p.src.size:.3e} pairs, {dt1:.1f} s, 1 thread"}
    check = {"max_rel_l2_fp32c_vs_oracle": errs, "points": int(len(sub)), "times": len(times)}
    return base, check


def config_errors(dev):
    """Part of the oracle leg: rel-L2 of every GPU precision against the FP64
    oracle, worst over the evaluation times, on the moving-charge workload
    (16^3 sources x 16^3 points, 4 times) and the dipole workload (32^3
    sources x 4096 points on shells, 4 times; worst shell)."""
    import torch

    import oracle
    import paper_2104_05426_gb300 as jefi
    from workloads import c1_lienard_wiechert, c3_dipole

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    out = {}
    for name, p in (("moving charge 16^3 x 16^3", c1_lienard_wiechert()),
                     ("dipole 32^3 x 4096 points", c3_dipole())):
        rho, J, _, _ = p.source.history(p.src, p.n_push, p.dt, p.t0)
        obs = p.obs()
        ref = [oracle.fields(p.src.n, p.src.lo, p.src.d, obs, rho, J, c=p.c, k_e=p.k_e, k_b=p.k_b,
                             dt=p.dt, t0=p.t0, t=t) for t in p.times]
        if p.obs_grid is None:
            r = np.linalg.norm(obs, axis=1)
            parts = [np.abs(r - R) < 1e-6 * R for R in np.unique(np.round(r, 6))]
        else:
            parts = [np.ones(len(obs), dtype=bool)]
        res = {}
        for prec in ("fp64", "fp32c", "fp32"):
            prm = jefi.default_params(c=p.c, k_e=p.k_e, k_b=p.k_b, dt=p.dt, t0=p.t0, history_slots=p.H,
                                      precision=prec)
            src = jefi.grid_from(p.src)
            h = (jefi.jefi_create(src, obs_grid=jefi.grid_from(p.obs_grid), params=prm)
                 if p.obs_grid is not None else jefi.jefi_create(src, obs_points=obs, params=prm))
            for n in range(p.n_push):
                jefi.jefi_push_sources(h, torch.from_numpy(np.ascontiguousarray(rho[n])).to(dev),
                                       torch.from_numpy(np.ascontiguousarray(J[n])).to(dev))
            E, B = jefi.eval_fields(h, list(p.times))
            E, B = E.cpu().numpy(), B.cpu().numpy()
            res[prec] = {f: max(rel(A[i][m], ref[i][k][m]) for i in range(len(p.times)) for m in parts)
                         for k, (f, A) in enumerate((("E", E), ("B", B)))}
            res[prec]["device_status"] = jefi.jefi_get_info(h)["device_status"]
            jefi.jefi_destroy(h)
        out[name] = res
    return out


# Published V100 timings of the paper: Table 2 (410 snapshots, 15^3 x 15^3,
# total GPU time, constant / sinusoidal sources) and Table 4 (GPU execution
# per time step at "ntg" = [n^3, n^3], lts = 500).  Context only: another GPU,
# unstated precision, and Table 4 likely includes per-call overheads.
PAPER_TABLE2_S = {"E1": 8.696, "E2": 8.111}
PAPER_TABLE4_S = {20: 1.001, 60: 2.720, 70: 4.858, 100: 32.565, 160: 521.970}


def paper_tables(sides=(20, 60, 70, 100, 160), lts=500, snapshots=410):
    """The paper's own timing workloads through the library (compensated FP32).

    Table 2: E1 (step-on constant) and E2 (sinusoidal) sources at the paper's
    sizes; per snapshot k = 0..409 one slice is pushed (from device memory)
    and E, B are evaluated at t = k dt, fields left on the device.  The ring
    holds 448 slices, more than E2's longest delay (416), so every snapshot
    sees its whole history.  Table 4: coincident n^3 grids over [-3,3]^3 with
    dt = d_m / lts (d_m the largest centre distance), lts + 8 resident slices
    of constant sources, one evaluation at the newest time (after one
    untimed)."""
    import torch

    import paper_2104_05426_gb300 as jefi
    from workloads import Grid, e1_constant, e2_sinusoidal

    dev = torch.device("cuda", 0)
    out = {"table2": {}, "table4": {}}
    for name, prob in (("E1", e1_constant()), ("E2", e2_sinusoidal())):
        H = 448
        prm = jefi.default_params(c=prob.c, k_e=prob.k_e, k_b=prob.k_b, dt=prob.dt, t0=prob.t0,
                                  history_slots=H, precision="fp32c")
        h = jefi.jefi_create(jefi.grid_from(prob.src), obs_grid=jefi.grid_from(prob.obs_grid), params=prm,
                             torch_allocator=True)
        sl = [prob.source.sample(prob.src, prob.t0 + k * prob.dt, k) for k in range(snapshots)]
        rho = torch.from_numpy(np.stack([r for r, _ in sl])).to(dev)
        J = torch.from_numpy(np.stack([j for _, j in sl])).to(dev)
        E = torch.empty((snapshots, prob.n_obs, 3), dtype=torch.float64, device=dev)
        B = torch.empty_like(E)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for k in range(snapshots):
            jefi.jefi_push_sources(h, rho[k], J[k])
            jefi.jefi_eval_fields(h, prob.t0 + k * prob.dt, E[k], B[k])
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        pairs = prob.src.size * prob.n_obs * snapshots
        out["table2"][name] = {"snapshots": snapshots, "total_s": ms / 1e3, "pairs_per_s": pairs / (ms / 1e3),
                               "paper_v100_total_s": PAPER_TABLE2_S[name],
                               "device_status": jefi.jefi_get_info(h)["device_status"]}
        jefi.jefi_destroy(h)
    for n in sides:
        g = Grid.cube(n, -3.0, 3.0)
        d_m = math.sqrt(3.0) * (6.0 - g.d[0])
        dt = d_m / lts
        H = lts + 8
        prm = jefi.default_params(dt=dt, history_slots=H, precision="fp32c")
        h = jefi.jefi_create(jefi.grid_from(g), obs_grid=jefi.grid_from(g), params=prm, torch_allocator=True)
        rho = torch.ones(g.size, dtype=torch.float64, device=dev)
        J = torch.ones((g.size, 3), dtype=torch.float64, device=dev)
        for _ in range(H):
            jefi.jefi_push_sources(h, rho, J)
        t = (H - 1) * dt
        E = torch.empty((g.size, 3), dtype=torch.float64, device=dev)
        B = torch.empty_like(E)
        jefi.jefi_eval_fields(h, t, E, B)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        jefi.jefi_eval_fields(h, t, E, B)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        info = jefi.jefi_get_info(h)
        out["table4"][str(n)] = {"lts": lts, "step_s": ms / 1e3, "pairs_per_s": g.size * g.size / (ms / 1e3),
                                 "staged_band": info["staged_band"], "paper_v100_step_s": PAPER_TABLE4_S.get(n),
                                 "device_status": info["device_status"]}
        jefi.jefi_destroy(h)
        del rho, J, E, B
        torch.cuda.empty_cache()
    return out


def run_reference(args):
    """Reference arm: the FP64 CPU oracle, as it stands, on the host cores."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from workloads import c2_heavy_ion

    p = c2_heavy_ion()
    slices = [p.source.sample(p.src, p.t0 + n * p.dt, n) for n in range(p.H)]
    rho = np.stack([s[0] for s in slices])
    J = np.stack([s[1] for s in slices])
    times = p.times
    stride = 4096
    sub = np.arange(0, p.n_obs, stride)
    obs = p.obs()[sub]

    def step():
        for t in times:
            oracle.fields(p.src.n, p.src.lo, p.src.d, obs, rho, J, dt=p.dt, t0=p.t0, t=t)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt_s = time.perf_counter() - t0
    pairs_step = len(sub) * p.src.size * len(times)
    value = pairs_step * args.steps / dt_s
    cores = oracle.max_threads()
    sample = (f"every {stride}th of {p.n_obs} observation points x {p.src.size} sources x "
              f"{len(times)} times = {pairs_step:.3e} pairs per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt_s * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "heavy-ion 64^3 src x 64^3 obs over [-5,5]^3, H=128, 8 eval times",
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
        flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="jefi", choices=["jefi", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 and oracle legs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--serving-c5", action="store_true",
                    help="only run the serving configuration (64 problems, --serving-requests per load "
                         "level at 0.5/0.8/1.0x saturation, 64 GB budget) with an oracle check of a "
                         "sample of served requests, and print it")
    ap.add_argument("--serving-requests", type=int, default=10000)
    ap.add_argument("--leg", default=None, choices=["dipole", "batch"],
                    help="only run one leg (the dipole workload, or the 256-problem batch) and print it "
                         "(for profiler captures of its kernels)")
    ap.add_argument("--batch-problems", type=int, default=256, help="problems of the --leg batch run")
    ap.add_argument("--paper-tables", action="store_true",
                    help="only time the paper's own workloads (Tables 2 and 4) and print them")
    ap.add_argument("--precision", default="fp32c", choices=["fp32c", "fp32", "fp64"],
                    help="precision of the timed path (fp32c = the benchmark; the others for "
                         "profiler captures and comparisons)")
    ap.add_argument("--side", type=int, default=64,
                    help="grid side of the heavy-ion workload (64 = the benchmark; smaller "
                         "sides only for profiler captures)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.leg == "dipole":
        import torch

        print(json.dumps(dipole_leg(torch.device("cuda", 0)), default=float))
    elif args.leg == "batch":
        from paper_2104_05426_gb300.serving import measure_batch

        r = measure_batch(n_problems=args.batch_problems, reps=1)
        print(json.dumps({k: r[k] for k in ("problems", "pairs", "ms_per_batch", "pairs_per_s", "by_kernel")},
                         default=float))
    elif args.paper_tables:
        print(json.dumps(paper_tables()))
    elif args.serving_c5:
        from paper_2104_05426_gb300.serving import measure

        res, samples = measure(n_requests=args.serving_requests, n_samples=8)
        res["oracle_check"] = served_oracle_check(samples, point_stride=31)
        print(json.dumps(res))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
