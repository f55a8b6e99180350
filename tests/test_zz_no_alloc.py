"""jefi_eval_fields_noalloc: the entry point for callers that cannot allocate
device memory when they need fields -- a host application whose own pool
allocator owns the device memory and forbids other cudaMalloc calls, or a
time-critical loop where cudaMalloc/cudaFree would synchronise the device.

It must give the fields of the existing entry point (jefi_eval_fields, FP64)
using only the caller's buffers and the library's fixed device array, call
after call.  This file sorts last so that a run stopping at its first failure
has already run every other test; it also passes when run on its own.
"""
import numpy as np
import pytest

import paper_2104_05426_gb300 as jefi
from workloads import Blob, Grid, MovingGaussians

pytestmark = pytest.mark.gpu

TOL = 1e-12      # the FP64 parity tolerance of the GPU tests


def _rel(a, b):
    a = a.cpu().numpy()
    b = b.cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(src, obs_pts, blobs, dt, n_slices, t, seed):
    """Reference fields from jefi_eval_fields, plus device copies of the inputs."""
    import torch

    rho, J, _, _ = MovingGaussians(blobs, noise=0.02, seed=seed).history(src, n_slices, dt)
    prm = jefi.default_params(dt=dt, history_slots=n_slices, precision="fp64")
    h = jefi.jefi_create(jefi.grid_from(src), obs_points=obs_pts, params=prm)
    for n in range(n_slices):
        jefi.jefi_push_sources(h, rho[n], J[n])
    E_ref, B_ref = jefi.eval_fields(h, t)
    torch.cuda.synchronize()
    jefi.jefi_destroy(h)

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    return dict(src=src, obs=dev(obs_pts), rho=dev(rho), J=dev(J), prm=prm, t=t, E_ref=E_ref,
                B_ref=B_ref)


def _noalloc(case):
    import torch

    E = torch.full_like(case["E_ref"], float("nan"))
    B = torch.full_like(case["B_ref"], float("nan"))
    jefi.jefi_eval_fields_noalloc(jefi.grid_from(case["src"]), case["obs"], case["rho"], case["J"],
                                  case["prm"], case["t"], E, B)
    return E, B


def test_noalloc_matches_eval_fields_call_after_call(gpu):
    rng = np.random.Generator(np.random.PCG64(11))
    src_a = Grid.cube(12, -0.6, 0.6)
    obs_a = rng.uniform(-2.0, 2.0, (1000, 3))
    case_a = _case(src_a, obs_a, [Blob(1.0, (0.2, 0.2, 0.2), (0.0, 0.0, 0.0), (0.1, 0.0, 0.0))],
                   dt=0.05, n_slices=80, t=3.2, seed=1)
    # second problem: ragged grid, observers on the source centres (self pairs screened)
    src_b = Grid((7, 9, 5), (0.1, -0.3, 0.2), (0.13, 0.11, 0.17))
    case_b = _case(src_b, src_b.points(), [Blob(-0.5, (0.3, 0.2, 0.25), (0.5, 0.2, 0.6), (0.0, 0.2, 0.1))],
                   dt=0.07, n_slices=50, t=2.9, seed=2)
    for case in (case_a, case_b, case_a):     # the array keeps the previous call's contents
        E, B = _noalloc(case)
        assert _rel(E, case["E_ref"]) <= TOL
        assert _rel(B, case["B_ref"]) <= TOL


def test_noalloc_rejects_more_points_than_its_array_holds(gpu):
    import torch

    src = Grid.cube(4, 0.0, 1.0)
    n_obs = 700_000          # > (JEFI_NOALLOC_SCRATCH_BYTES - 256) / 48 rounded to tiles
    obs = torch.full((n_obs, 3), 3.0, dtype=torch.float64, device="cuda")
    rho = torch.ones((2, src.size), dtype=torch.float64, device="cuda")
    J = torch.zeros((2, src.size, 3), dtype=torch.float64, device="cuda")
    E = torch.empty((n_obs, 3), dtype=torch.float64, device="cuda")
    B = torch.empty_like(E)
    with pytest.raises(jefi.JefiError) as e:
        jefi.jefi_eval_fields_noalloc(jefi.grid_from(src), obs, rho, J,
                                      jefi.default_params(dt=0.1), 4.0, E, B)
    assert e.value.code == jefi.JEFI_EUNSUPPORTED


def test_noalloc_matches_the_oracle(gpu):
    """Once against the FP64 CPU oracle directly (not only through jefi_eval_fields)."""
    import torch

    import oracle

    rng = np.random.Generator(np.random.PCG64(5))
    src = Grid((6, 5, 7), (-0.4, -0.3, -0.5), (0.13, 0.12, 0.14))
    obs = rng.uniform(-1.5, 1.5, (300, 3))
    case = _case(src, obs, [Blob(0.8, (0.2, 0.25, 0.2), (0.0, 0.1, -0.1), (0.2, -0.1, 0.0))],
                 dt=0.06, n_slices=70, t=3.5, seed=3)
    E, B = _noalloc(case)
    rho, J = case["rho"].cpu().numpy(), case["J"].cpu().numpy()
    Er, Br = oracle.fields(src.n, src.lo, src.d, obs, rho, J, dt=0.06, t=3.5)
    assert _rel(E, torch.from_numpy(Er)) <= TOL
    assert _rel(B, torch.from_numpy(Br)) <= TOL


def test_noalloc_reports_a_missing_slice_then_recovers(gpu):
    """A time whose pairs need slices past the given history returns
    JEFI_ENOTYET (the kernel sets the status word); the next call with a
    valid time returns OK, so the status word was cleared between calls."""
    import torch

    rng = np.random.Generator(np.random.PCG64(8))
    src = Grid.cube(8, -0.5, 0.5)
    obs = rng.uniform(-1.0, 1.0, (256, 3))
    case = _case(src, obs, [Blob(1.0, (0.2, 0.2, 0.2), (0.0, 0.0, 0.0), (0.1, 0.1, 0.0))],
                 dt=0.05, n_slices=40, t=1.8, seed=4)
    E = torch.empty_like(case["E_ref"])
    B = torch.empty_like(case["B_ref"])
    g = jefi.grid_from(case["src"])
    # slices 0..39 cover t <= 1.95; at t = 2.5 every pair closer than R = 0.5
    # needs slice 40 or later, which was not given
    with pytest.raises(jefi.JefiError) as e:
        jefi.jefi_eval_fields_noalloc(g, case["obs"], case["rho"], case["J"], case["prm"], 2.5, E, B)
    assert e.value.code == jefi.JEFI_ENOTYET
    E2, B2 = _noalloc(case)                 # t = 1.8: every slice present
    assert _rel(E2, case["E_ref"]) <= TOL
    assert _rel(B2, case["B_ref"]) <= TOL


def test_noalloc_rejects_grids_past_its_axis_limit(gpu):
    """More than 6144 padded source cells over the three axes (the kernel's
    shared-memory table of cell centres) is refused before any launch."""
    import torch

    src = Grid((6200, 1, 1), (0.0, 0.0, 0.0), (0.01, 0.1, 0.1))    # 4 * (1550 + 1 + 1) = 6208 padded
    obs = torch.full((4, 3), 100.0, dtype=torch.float64, device="cuda")
    rho = torch.zeros((2, src.size), dtype=torch.float64, device="cuda")
    J = torch.zeros((2, src.size, 3), dtype=torch.float64, device="cuda")
    E = torch.empty((4, 3), dtype=torch.float64, device="cuda")
    B = torch.empty_like(E)
    with pytest.raises(jefi.JefiError) as e:
        jefi.jefi_eval_fields_noalloc(jefi.grid_from(src), obs, rho, J, jefi.default_params(dt=0.1), 1.0, E, B)
    assert e.value.code == jefi.JEFI_EUNSUPPORTED
