"""Shared helpers of the GPU tests: run a workloads.Problem through the oracle
and through libjefi on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2104_05426_gb300 as jefi


def history(problem, n_slices=None):
    n = problem.n_push if n_slices is None else n_slices
    return problem.source.history(problem.src, n, problem.dt, problem.t0)


def oracle_fields(problem, hist, times, supplied=False, screen=None, with_abs=False):
    rho, J, drho, dJ = hist
    kw = dict(drho=drho, dJ=dJ) if supplied else {}
    out = []
    for t in times:
        out.append(oracle.fields(problem.src.n, problem.src.lo, problem.src.d, problem.obs(), rho, J,
                                 c=problem.c, k_e=problem.k_e, k_b=problem.k_b, dt=problem.dt,
                                 t0=problem.t0, t=t, screen=screen, with_abs=with_abs, **kw))
    return out


def create(problem, precision, H=None, supplied=False, screen=None, flags=0, torch_allocator=False):
    kw = dict(c=problem.c, k_e=problem.k_e, k_b=problem.k_b, dt=problem.dt, t0=problem.t0,
              history_slots=problem.H if H is None else H, precision=precision, flags=flags,
              deriv=jefi.JEFI_DERIV_SUPPLIED if supplied else jefi.JEFI_DERIV_BACKWARD)
    if screen is not None:
        kw["screen"] = screen
    p = jefi.default_params(**kw)
    src = jefi.grid_from(problem.src)
    if problem.obs_grid is not None:
        return jefi.jefi_create(src, obs_grid=jefi.grid_from(problem.obs_grid), params=p,
                                torch_allocator=torch_allocator)
    return jefi.jefi_create(src, obs_points=problem.obs_points, params=p,
                            torch_allocator=torch_allocator)


def push_all(h, hist, supplied=False, device=True, upto=None):
    import torch

    rho, J, drho, dJ = hist
    n = rho.shape[0] if upto is None else upto
    for i in range(n):
        args = [rho[i], J[i]]
        if supplied:
            args += [drho[i], dJ[i]]
        if device:
            args = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in args]
        jefi.jefi_push_sources(h, *args)


def gpu_fields(h, times):
    E, B = jefi.eval_fields(h, np.asarray(times, dtype=np.float64))
    return E.cpu().numpy(), B.cpu().numpy()


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))
