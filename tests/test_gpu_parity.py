"""GPU parity of libjefi against the FP64 oracle (through the C ABI).

Tolerances (stated per field, normwise over all points and times):
  * retarded slots: identical to the oracle's for every pair;
  * FP64 path: rel-L2 <= 1e-12;
  * compensated FP32 path: rel-L2 <= 1e-5 on physical workloads; on random
    (cancelling) sources the error is measured against the norm of the
    oracle's sum of |term| (a per-term rounding bound): <= 5e-6 there.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2104_05426_gb300 as jefi
from jefi_cases import create, gpu_fields, history, oracle_fields, push_all, rel_l2
from workloads import (Blob, Dipole, Grid, MovingGaussians, Problem, c1_lienard_wiechert,
                       c2_heavy_ion, shell_points)

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32C_TOL = 1e-5


@pytest.fixture(scope="module")
def c1():
    p = c1_lienard_wiechert()
    hist = history(p)
    ref = oracle_fields(p, hist, p.times)
    return p, hist, ref


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32c", FP32C_TOL), ("fp32", 3e-5)])
def test_c1_fields_match_oracle(gpu, c1, prec, tol):
    p, hist, ref = c1
    h = create(p, prec)
    push_all(h, hist)
    E, B = gpu_fields(h, p.times)
    for i in range(len(p.times)):
        assert rel_l2(E[i], ref[i][0]) <= tol, (prec, i, rel_l2(E[i], ref[i][0]))
        assert rel_l2(B[i], ref[i][1]) <= tol, (prec, i, rel_l2(B[i], ref[i][1]))
    info = jefi.jefi_get_info(h)
    assert info["device_status"] == 0
    if prec != "fp64":
        assert info["staged_band"] > 0          # 16^3 lattice grids take the staged kernel
    jefi.jefi_destroy(h)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_c1_slots_bit_exact(gpu, c1, prec):
    p, hist, _ = c1
    h = create(p, prec)
    push_all(h, hist)
    for t in p.times:
        got = jefi.jefi_debug_slots(h, t)
        ref = oracle.all_slots(p.src.n, p.src.lo, p.src.d, p.obs(), dt=p.dt, t0=p.t0, c=p.c, t=t)
        scr = ref == oracle.SCREENED
        assert np.array_equal(got[scr], np.full(scr.sum(), np.iinfo(np.int32).min))
        assert np.array_equal(got[~scr].astype(np.int64), ref[~scr])
    jefi.jefi_destroy(h)


def test_multi_time_equals_single_time_and_host_io(gpu, c1):
    p, hist, _ = c1
    h = create(p, "fp32c")
    push_all(h, hist)
    Em, Bm = gpu_fields(h, p.times)
    for i, t in enumerate(p.times):
        E1 = np.empty((p.n_obs, 3))
        B1 = np.empty((p.n_obs, 3))
        jefi.jefi_eval_fields(h, t, E1, B1)          # host outputs
        assert np.array_equal(E1, Em[i]) and np.array_equal(B1, Bm[i])
    jefi.jefi_destroy(h)


def _random_problem(src_n, obs_n, coincide, seed, H=40, dt=0.05):
    rng = np.random.Generator(np.random.PCG64(seed))
    d = 0.1
    src = Grid(tuple(src_n), (-0.63, -0.41, -0.37), (d, d * 1.1, d * 0.9))
    if coincide:
        obs = Grid(tuple(obs_n), src.lo, src.d)      # same lattice: self cells screened
    else:
        obs = Grid(tuple(obs_n), (0.91, -0.2, 0.15), (0.07, 0.05, 0.11))
    prob = Problem("rand", src, obs, None, dt, H, H, [], MovingGaussians([]))
    rho = rng.standard_normal((H, src.size))
    J = rng.standard_normal((H, src.size, 3))
    return prob, (rho, J, None, None)


@pytest.mark.parametrize("coincide", [True, False])
def test_ragged_grids_with_screening(gpu, coincide):
    """Grid extents that are not multiples of the 4^3 brick or the 8x8x4
    tile, overlapping (screened) or disjoint, random histories."""
    prob, hist = _random_problem((13, 10, 7), (11, 9, 6), coincide, seed=21)
    rmax = math.sqrt(sum((n * d + 1.5) ** 2 for n, d in zip(prob.src.n, prob.src.d)))
    times = [prob.t0 + (prob.H - 1) * prob.dt - 0.013, 1.2345]
    times = [t for t in times if t > 0]
    ref = oracle_fields(prob, hist, times, with_abs=True)
    for prec, tol in (("fp64", 2e-14), ("fp32c", 5e-6)):
        h = create(prob, prec)
        push_all(h, hist)
        E, B = gpu_fields(h, times)
        for i in range(len(times)):
            Er, Br, aE, aB = ref[i]
            assert np.linalg.norm(E[i] - Er) <= tol * np.linalg.norm(aE), (prec, i)
            assert np.linalg.norm(B[i] - Br) <= tol * np.linalg.norm(aB), (prec, i)
            got = jefi.jefi_debug_slots(h, times[i])
            rs = oracle.all_slots(prob.src.n, prob.src.lo, prob.src.d, prob.obs(), dt=prob.dt,
                                  t0=prob.t0, t=times[i])
            sc = rs == oracle.SCREENED
            assert np.array_equal(got[~sc].astype(np.int64), rs[~sc])
            assert np.all(got[sc] == np.iinfo(np.int32).min)
            if coincide:
                assert sc.sum() >= prob.n_obs       # every point screens its own cell
        assert jefi.jefi_get_info(h)["device_status"] == 0
        jefi.jefi_destroy(h)


def test_point_list_dipole_supplied_derivatives(gpu):
    """Explicit observation points (Morton-tiled), supplied derivatives,
    c != 1 and k_e != k_b."""
    src = Grid.cube(12, -0.5, 0.5)
    pts = shell_points([3.0, 6.0], 300, seed=5)
    model = Dipole(1.0, 2 * math.pi / 8.0, 0.1)
    c, dt, H = 2.0, 0.05, 96
    t0 = -(6.9 / c + 2 * dt)
    prob = Problem("dip", src, None, pts, dt, H, H, [], model, c=c, k_e=0.7, k_b=0.7 / c ** 2, t0=t0)
    hist = history(prob)
    t_hi = t0 + (H - 1) * dt + 2.1 / c
    times = [t_hi - 0.3, t_hi - 0.01]
    ref = oracle_fields(prob, hist, times, supplied=True)
    for prec, tol in (("fp64", FP64_TOL), ("fp32c", FP32C_TOL)):
        h = create(prob, prec, supplied=True)
        push_all(h, hist, supplied=True, device=False)   # host inputs
        E, B = gpu_fields(h, times)
        for i in range(len(times)):
            assert rel_l2(E[i], ref[i][0]) <= tol
            assert rel_l2(B[i], ref[i][1]) <= tol
        jefi.jefi_destroy(h)


def test_ring_wraparound_and_window(gpu):
    """Push 3.5x the ring size; evaluate inside the sliding window against
    the oracle run on the full history; just outside it is an error."""
    src = Grid.cube(6, -0.3, 0.3)
    obs = Grid.box((5, 4, 3), (1.0, -0.5, -0.2), (1.5, 0.5, 0.2))
    H, dt = 24, 0.05
    blob = Blob(1.0, (0.15,) * 3, (-0.2, 0.0, 0.0), (0.05, 0.02, 0.0))
    prob = Problem("wrap", src, obs, None, dt, H, 84, [], MovingGaussians([blob], noise=0.05, seed=9))
    hist = history(prob)
    for prec, tol in (("fp64", FP64_TOL), ("fp32c", FP32C_TOL)):
        h = create(prob, prec)
        push_all(h, hist)
        lo, hi = jefi.jefi_valid_window(h)
        assert lo < hi
        times = [lo, 0.5 * (lo + hi), hi]
        ref = oracle_fields(prob, hist, times)
        E, B = gpu_fields(h, times)
        for i in range(3):
            assert rel_l2(E[i], ref[i][0]) <= tol and rel_l2(B[i], ref[i][1]) <= tol
        with pytest.raises(jefi.JefiError) as e:
            jefi.eval_fields(h, np.nextafter(hi, math.inf) + 1e-9)
        assert e.value.code == jefi.JEFI_ENOTYET
        with pytest.raises(jefi.JefiError) as e:
            jefi.eval_fields(h, lo - 2 * dt)
        assert e.value.code == jefi.JEFI_EEVICTED
        jefi.jefi_destroy(h)


def test_exact_ties_dyadic_geometry(gpu):
    """Dyadic grids and times where many pairs sit exactly on a slot
    boundary: every precision selects the oracle's slot."""
    src = Grid((8, 8, 8), (-1.0, -1.0, -1.0), (0.25, 0.25, 0.25))
    obs = Grid((8, 8, 4), (-1.0, -1.0, 1.0), (0.25, 0.25, 0.25))
    dt, H = 0.125, 64
    prob = Problem("ties", src, obs, None, dt, H, H, [], MovingGaussians([]))
    rng = np.random.Generator(np.random.PCG64(4))
    hist = (rng.standard_normal((H, src.size)), rng.standard_normal((H, src.size, 3)), None, None)
    times = [6.0, 6.125, 5.5 + 0.125 * 3]          # T/dt integer: R = k*dt ties are exact
    for prec in ("fp64", "fp32c", "fp32"):
        h = create(prob, prec)
        push_all(h, hist)
        for t in times:
            got = jefi.jefi_debug_slots(h, t)
            ref = oracle.all_slots(src.n, src.lo, src.d, obs.points(), dt=dt, t=t)
            sc = ref == oracle.SCREENED
            assert np.array_equal(got[~sc].astype(np.int64), ref[~sc]), prec
        jefi.jefi_destroy(h)


@pytest.mark.parametrize("flags", [0, jefi.JEFI_FLAG_DIRECT_GATHER])
def test_non_lattice_exact_ties_slots(gpu, flags):
    """Decimal (non-dyadic) lattices with offsets that are exact multiples of
    c dt in real arithmetic (axis offsets k 0.1, Pythagorean (0.3, 0.4, 0)
    ...), evaluated at multiples of dt: many pairs sit on a slot boundary of
    the FP64 rule, so the FP32 kernels leave them undecided, and their
    double-float check must defer to the FP64 rule (it cannot separate S
    from the threshold).  Slots identical to the oracle's; batched results
    bit-identical to single evaluations."""
    import torch

    src = Grid((10, 10, 10), (0.0, 0.0, 0.0), (0.1, 0.1, 0.1))
    obs = Grid((10, 10, 6), (0.0, 0.0, 1.2), (0.1, 0.1, 0.1))
    dt, H = 0.05, 96
    prob = Problem("decimal ties", src, obs, None, dt, H, H, [], MovingGaussians([]))
    rng = np.random.Generator(np.random.PCG64(12))
    hist = (rng.standard_normal((H, src.size)), rng.standard_normal((H, src.size, 3)), None, None)
    h = create(prob, "fp32c", flags=flags | jefi.JEFI_FLAG_STATS)
    push_all(h, hist)
    info = jefi.jefi_get_info(h)
    assert (info["staged_band"] > 0) == (flags == 0)
    lo, hi = jefi.jefi_valid_window(h)
    k_hi = math.floor(hi / dt)
    times = [k * dt for k in (k_hi, k_hi - 3) if k * dt >= lo]
    assert times
    for t in times:
        got = jefi.jefi_debug_slots(h, t)
        ref = oracle.all_slots(src.n, src.lo, src.d, obs.points(), dt=dt, t=t)
        sc = ref == oracle.SCREENED
        assert np.array_equal(got[~sc].astype(np.int64), ref[~sc]), t
    jefi.jefi_reset_stats(h)
    E1 = torch.empty((obs.size, 3), dtype=torch.float64, device="cuda")
    B1 = torch.empty_like(E1)
    jefi.jefi_eval_fields(h, times[0], E1, B1)
    assert jefi.jefi_get_info(h)["slot_fallbacks"] > 0      # the geometry does leave pairs undecided
    E2, B2 = torch.empty_like(E1), torch.empty_like(E1)
    jefi.jefi_eval_batch([h], [times[0]], [E2], [B2])
    torch.cuda.synchronize()
    assert torch.equal(E1, E2) and torch.equal(B1, B2)
    assert jefi.jefi_get_info(h)["device_status"] == 0
    jefi.jefi_destroy(h)


def test_random_non_lattice_geometry_slots(gpu):
    """Non-dyadic spacings, offsets, c and dt with scattered points: the
    FP32 path's guarded slot selection still matches on ~3e7 pairs."""
    rng = np.random.Generator(np.random.PCG64(8))
    src = Grid((20, 17, 23), (-0.731, 0.113, -1.317), (0.0931, 0.1077, 0.0853))
    pts = rng.uniform(-3.0, 3.0, (4000, 3))
    c, dt, H = 1.37, 0.0173, 700
    prob = Problem("nl", src, None, pts, dt, H, H, [], MovingGaussians([]), c=c)
    hist = (np.zeros((H, src.size)), np.zeros((H, src.size, 3)), None, None)
    h = create(prob, "fp32c", flags=jefi.JEFI_FLAG_STATS)
    push_all(h, hist, device=False)
    lo, hi = jefi.jefi_valid_window(h)
    for t in (hi, hi - 0.377):
        got = jefi.jefi_debug_slots(h, t)
        ref = oracle.all_slots(src.n, src.lo, src.d, pts, dt=dt, t=t, c=c)
        sc = ref == oracle.SCREENED
        assert np.array_equal(got[~sc].astype(np.int64), ref[~sc])
    jefi.jefi_destroy(h)


def test_degenerate_inputs(gpu):
    """No observation points; a source grid with a zero extent; every pair
    screened; a single source cell."""
    src = Grid.cube(4, 0.0, 1.0)
    p = jefi.default_params(dt=0.1, history_slots=8)
    h = jefi.jefi_create(jefi.grid_from(src), obs_points=np.zeros((0, 3)), params=p)
    jefi.jefi_push_sources(h, np.ones(64), np.ones((64, 3)))
    E = np.empty((0, 3))
    jefi.jefi_eval_fields(h, 0.5, E, E.copy())
    jefi.jefi_destroy(h)
    # zero extent: no sources at all -> zero fields
    h = jefi.jefi_create(jefi.grid((0, 4, 4), (0, 0, 0), (0.25,) * 3), obs_points=np.ones((7, 3)),
                         params=p)
    jefi.jefi_push_sources(h, np.zeros(0), np.zeros((0, 3)))
    E, B = jefi.eval_fields(h, 0.3)
    assert float(E.abs().max()) == 0.0 and float(B.abs().max()) == 0.0
    jefi.jefi_destroy(h)
    # every pair screened (one cell, observer at its centre)
    one = Grid.cube(1, 0.0, 1.0)
    for prec in ("fp64", "fp32c"):
        q = jefi.default_params(dt=0.1, history_slots=8, precision=prec)
        h = jefi.jefi_create(jefi.grid_from(one), obs_points=[[0.5, 0.5, 0.5]], params=q)
        jefi.jefi_push_sources(h, np.ones(1), np.ones((1, 3)))
        E, B = jefi.eval_fields(h, 0.05)
        assert float(E.abs().max()) == 0.0
        jefi.jefi_destroy(h)
        # a single cell seen from outside: Coulomb + Biot-Savart of the static part
        h = jefi.jefi_create(jefi.grid_from(one), obs_points=[[2.5, 0.5, 0.5]], params=q)
        for _ in range(8):
            jefi.jefi_push_sources(h, np.full(1, 2.0), np.array([[0.0, 1.0, 0.0]]))
        E, B = jefi.eval_fields(h, 2.75)           # R = 2: slot 7, past the turn-on slice
        np.testing.assert_allclose(E.cpu().numpy(), [[2.0 / 4.0, 0, 0]], rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(B.cpu().numpy(), [[0, 0, -1.0 / 4.0]], rtol=1e-6, atol=1e-12)
        jefi.jefi_destroy(h)


def test_invalid_arguments(gpu):
    g = jefi.grid((4, 4, 4), (0, 0, 0), (0.25,) * 3)
    for bad in (dict(dt=0.0), dict(c=-1.0), dict(history_slots=0), dict(precision=7)):
        p = jefi.default_params(**{**dict(dt=0.1), **bad})
        with pytest.raises(jefi.JefiError) as e:
            jefi.jefi_create(g, obs_points=np.ones((3, 3)) * 2, params=p)
        assert e.value.code == jefi.JEFI_EINVAL
    with pytest.raises(jefi.JefiError):
        jefi.jefi_create(g, obs_points=np.array([[np.nan, 0, 0]]), params=jefi.default_params(dt=0.1))
    h = jefi.jefi_create(g, obs_points=np.ones((3, 3)) * 2, params=jefi.default_params(dt=0.1))
    with pytest.raises(jefi.JefiError) as e:      # nothing pushed yet
        jefi.eval_fields(h, 5.0)
    assert e.value.code == jefi.JEFI_ENOTYET
    with pytest.raises(jefi.JefiError):           # derivatives given in backward mode
        jefi.jefi_push_sources(h, np.ones(64), np.ones((64, 3)), np.ones(64), np.ones((64, 3)))
    jefi.jefi_destroy(h)


def test_c2_full_size_sampled(gpu):
    """64^3 x 64^3 heavy-ion workload at full size, in the launch
    configuration the benchmark times (all 8 times in one call): FP32c and
    FP64 against the oracle on every 512th observation point."""
    p = c2_heavy_ion()
    h32 = create(p, "fp32c")
    h64 = create(p, "fp64")
    import torch

    for n in range(p.n_push):
        rho, J = p.source.sample(p.src, p.t0 + n * p.dt, n)
        r, j = torch.from_numpy(rho).cuda(), torch.from_numpy(J).cuda()
        jefi.jefi_push_sources(h32, r, j)
        jefi.jefi_push_sources(h64, r, j)
    E32, B32 = gpu_fields(h32, p.times)
    t_check = [p.times[0], p.times[-1]]
    E64, B64 = gpu_fields(h64, t_check)
    sub = np.arange(0, p.n_obs, 512)
    hist = history(p)
    obs = p.obs()[sub]
    for k, ti in enumerate((0, len(p.times) - 1)):
        Er, Br = oracle.fields(p.src.n, p.src.lo, p.src.d, obs, hist[0], hist[1], dt=p.dt,
                               t=p.times[ti])
        assert rel_l2(E32[ti][sub], Er) <= FP32C_TOL
        assert rel_l2(B32[ti][sub], Br) <= FP32C_TOL
        assert rel_l2(E64[k][sub], Er) <= FP64_TOL
        assert rel_l2(B64[k][sub], Br) <= FP64_TOL
    # the compensated path on every point against the FP64 GPU path
    assert rel_l2(E32[0], E64[0]) <= FP32C_TOL and rel_l2(B32[0], B64[0]) <= FP32C_TOL
    jefi.jefi_destroy(h32)
    jefi.jefi_destroy(h64)


@pytest.mark.parametrize("lattice", [True, False])
def test_staged_kernel_matches_direct_gather(gpu, lattice):
    """The TMA-staged FP32 kernel and the direct-gather FP32 kernel are two
    implementations of the same sum: identical slots for every pair, fields
    equal to FP32 rounding, both within tolerance of the oracle.  On an exact
    lattice the staged kernel decides every slot without an FP64 fall-back."""
    if lattice:
        src = Grid.cube(16, -1.0, 1.0)
        obs = Grid.box((16, 16, 8), (1.5, -1.0, -0.5), (3.5, 1.0, 0.5))
        dt = 0.0625
    else:
        src = Grid((16, 16, 16), (-0.731, -0.683, -0.802), (0.0931, 0.0877, 0.1013))
        obs = Grid((16, 16, 8), (1.113, -0.917, -0.419), (0.1207, 0.1133, 0.1049))
        dt = 0.0517
    blob = Blob(1.0, (0.25, 0.2, 0.3), (-0.2, 0.05, 0.0), (0.2, 0.1, -0.05))
    H = 120
    prob = Problem("st", src, obs, None, dt, H, H, [], MovingGaussians([blob], noise=0.02, seed=3))
    hist = history(prob)
    handles = {}
    for name, flags in (("staged", jefi.JEFI_FLAG_STATS),
                        ("direct", jefi.JEFI_FLAG_STATS | jefi.JEFI_FLAG_DIRECT_GATHER)):
        h = create(prob, "fp32c", flags=flags)
        push_all(h, hist)
        handles[name] = h
    info_s = jefi.jefi_get_info(handles["staged"])
    info_d = jefi.jefi_get_info(handles["direct"])
    assert info_s["staged_band"] > 0 and info_d["staged_band"] == 0
    lo, hi = jefi.jefi_valid_window(handles["staged"])
    times = [hi - 0.4, hi - 0.02]
    ref = oracle_fields(prob, hist, times)
    out = {k: gpu_fields(h, times) for k, h in handles.items()}
    for i, t in enumerate(times):
        s_st = jefi.jefi_debug_slots(handles["staged"], t)
        s_di = jefi.jefi_debug_slots(handles["direct"], t)
        assert np.array_equal(s_st, s_di)
        for k in out:
            assert rel_l2(out[k][0][i], ref[i][0]) <= FP32C_TOL
            assert rel_l2(out[k][1][i], ref[i][1]) <= FP32C_TOL
        assert rel_l2(out["staged"][0][i], out["direct"][0][i]) <= 2e-6
        assert rel_l2(out["staged"][1][i], out["direct"][1][i]) <= 2e-6
    info_s = jefi.jefi_get_info(handles["staged"])
    assert info_s["device_status"] == 0
    if lattice:
        assert info_s["slot_fallbacks"] == 0
    for h in handles.values():
        jefi.jefi_destroy(h)


def test_select_kernel_switches_and_measures(gpu):
    """jefi_select_kernel on a staged handle: switched to the direct gather it
    gives the slots and fields of a handle created on the direct gather, bit
    for bit; switched back, its own again; measuring keeps one of the two,
    and a batched evaluation follows the choice.  Handles without a staged
    band at creation and FP64 handles refuse."""
    import torch

    src = Grid((16, 16, 16), (-0.731, -0.683, -0.802), (0.0931, 0.0877, 0.1013))
    obs = Grid((16, 16, 8), (1.113, -0.917, -0.419), (0.1207, 0.1133, 0.1049))
    blob = Blob(1.0, (0.25, 0.2, 0.3), (-0.2, 0.05, 0.0), (0.2, 0.1, -0.05))
    prob = Problem("sel", src, obs, None, 0.0517, 120, 120, [], MovingGaussians([blob], noise=0.02, seed=3))
    hist = history(prob)
    hs = create(prob, "fp32c")
    hd = create(prob, "fp32c", flags=jefi.JEFI_FLAG_DIRECT_GATHER)
    for h in (hs, hd):
        push_all(h, hist)
    band0 = jefi.jefi_get_info(hs)["staged_band"]
    assert band0 > 0 and jefi.jefi_get_info(hd)["staged_band"] == 0
    lo, hi = jefi.jefi_valid_window(hs)
    times = [hi - 0.4, hi - 0.02]
    f_staged = gpu_fields(hs, times)
    f_direct = gpu_fields(hd, times)
    slots_d = [jefi.jefi_debug_slots(hd, t) for t in times]

    assert jefi.jefi_select_kernel(hs, jefi.JEFI_KERNEL_DIRECT) == 0
    assert jefi.jefi_get_info(hs)["staged_band"] == 0
    for a, b in zip(gpu_fields(hs, times), f_direct):
        assert np.array_equal(a, b)
    for t, sd in zip(times, slots_d):
        assert np.array_equal(jefi.jefi_debug_slots(hs, t), sd)

    assert jefi.jefi_select_kernel(hs, jefi.JEFI_KERNEL_STAGED) == band0
    for a, b in zip(gpu_fields(hs, times), f_staged):
        assert np.array_equal(a, b)

    band = jefi.jefi_select_kernel(hs, jefi.JEFI_KERNEL_MEASURE, times[0])
    # the creation band, the next wider compiled band, or the direct gather
    assert (band == 0 or band >= band0) and jefi.jefi_get_info(hs)["staged_band"] == band
    mine = gpu_fields(hs, times)
    if band in (0, band0):
        for a, b in zip(mine, f_direct if band == 0 else f_staged):
            assert np.array_equal(a, b)
    for t, sd in zip(times, slots_d):
        assert np.array_equal(jefi.jefi_debug_slots(hs, t), sd)
    E = torch.empty((prob.n_obs, 3), dtype=torch.float64, device="cuda")
    B = torch.empty_like(E)
    jefi.jefi_eval_batch([hs], [times[1]], [E], [B])
    torch.cuda.synchronize()
    assert np.array_equal(E.cpu().numpy(), mine[0][1]) and np.array_equal(B.cpu().numpy(), mine[1][1])
    ref = oracle_fields(prob, hist, times)
    for i in range(len(times)):
        assert rel_l2(mine[0][i], ref[i][0]) <= FP32C_TOL and rel_l2(mine[1][i], ref[i][1]) <= FP32C_TOL

    with pytest.raises(jefi.JefiError) as e:
        jefi.jefi_select_kernel(hd, jefi.JEFI_KERNEL_STAGED)
    assert e.value.code == jefi.JEFI_EUNSUPPORTED
    assert jefi.jefi_select_kernel(hd, jefi.JEFI_KERNEL_MEASURE, times[0]) == 0
    with pytest.raises(jefi.JefiError) as e:
        jefi.jefi_select_kernel(hs, jefi.JEFI_KERNEL_MEASURE, hi + 10.0)
    assert e.value.code != 0
    h64 = create(prob, "fp64")
    with pytest.raises(jefi.JefiError) as e:
        jefi.jefi_select_kernel(h64, jefi.JEFI_KERNEL_DIRECT)
    assert e.value.code == jefi.JEFI_EINVAL
    for h in (hs, hd, h64):
        assert jefi.jefi_get_info(h)["device_status"] == 0
        jefi.jefi_destroy(h)


def test_direct_gather_history_limit(gpu):
    """The direct-gather FP32 kernel packs two physical ring rows in 16 bits
    each: a handle on it whose ring has at most 65536 rows (the period H
    rounded up to a multiple of 4, plus the 4-slot zero line) is created,
    one more period step is refused with JEFI_EUNSUPPORTED (the FP64 path
    has no such limit)."""
    src = Grid.cube(4, -0.5, 0.5)
    obs = np.array([[3.0, 0.1, 0.2], [-2.5, 1.0, 0.3]])
    for H, ok in ((65532, True), (65533, False)):
        prm = jefi.default_params(dt=0.01, history_slots=H, precision="fp32c",
                                  flags=jefi.JEFI_FLAG_DIRECT_GATHER)
        if ok:
            h = jefi.jefi_create(jefi.grid_from(src), obs_points=obs, params=prm)
            assert jefi.jefi_get_info(h)["staged_band"] == 0
            jefi.jefi_destroy(h)
        else:
            with pytest.raises(jefi.JefiError) as e:
                jefi.jefi_create(jefi.grid_from(src), obs_points=obs, params=prm)
            assert e.value.code == jefi.JEFI_EUNSUPPORTED
    prm = jefi.default_params(dt=0.01, history_slots=65536, precision="fp64")
    jefi.jefi_destroy(jefi.jefi_create(jefi.grid_from(src), obs_points=obs, params=prm))


@pytest.mark.parametrize("src_side,dt,band", [(8, 0.2, 32), (16, 0.125, 48), (12, 0.12, 48), (10, 0.2, 32),
                                              (16, 0.065, 64), (12, 0.07, 64), (16, 0.045, 96), (10, 0.045, 96)])
def test_wide_band_staged_kernel(gpu, src_side, dt, band):
    """Coarse observation grids with fine time steps give slot bands of 32 to
    96 rows, which the staged kernel copies as 128-byte swizzled lines of 4
    slots in stages of two z slabs (32, 48) or one (64, 96): every slot
    bit-exact with the oracle and the fields within tolerance, on lattice
    (16^3, 8^3) and non-lattice (12^3, 10^3) source grids.  The band each
    case needs follows from the tile and brick extents: (2.59 + 5.20 d_src)
    / dt + 7 slots, plus 3 for the line alignment."""
    src = Grid.cube(src_side, -1.0, 1.0)
    obs = Grid.cube(16, -2.0, 2.0)
    blob = Blob(1.0, (0.25, 0.3, 0.2), (-0.1, 0.05, 0.0), (0.3, -0.1, 0.2))
    H = int(math.ceil(6.0 / dt)) + 8
    p = Problem("wide", src, obs, None, dt, H, H, [], MovingGaussians([blob], noise=0.02, seed=7))
    hist = history(p)
    h = create(p, "fp32c")
    push_all(h, hist)
    assert jefi.jefi_get_info(h)["staged_band"] == band
    _, hi = jefi.jefi_valid_window(h)
    times = [hi - 0.3, hi]
    ref = oracle_fields(p, hist, times)
    E, B = gpu_fields(h, times)
    for i, t in enumerate(times):
        assert rel_l2(E[i], ref[i][0]) <= FP32C_TOL
        assert rel_l2(B[i], ref[i][1]) <= FP32C_TOL
        got = jefi.jefi_debug_slots(h, t)
        want = oracle.all_slots(p.src.n, p.src.lo, p.src.d, p.obs(), dt=p.dt, t0=p.t0, c=p.c, t=t)
        scr = want == oracle.SCREENED
        assert np.array_equal(got[~scr].astype(np.int64), want[~scr])
    assert jefi.jefi_get_info(h)["device_status"] == 0
    jefi.jefi_destroy(h)


@pytest.mark.parametrize("shape", list(range(1, 10)))
def test_tile_shapes(gpu, shape):
    """Every observation tiling (the box shapes JEFI_TILE_8x8x4 ...
    JEFI_TILE_4x4x16 and JEFI_TILE_PACKED) on a ragged grid: slots bit-exact
    with the oracle and fields within tolerance; the automatic choice reports
    one of them."""
    src = Grid((14, 11, 9), (-0.7, -0.55, -0.45), (0.1, 0.1, 0.1))
    obs = Grid((19, 13, 11), (0.9, -0.8, -0.6), (0.11, 0.12, 0.1))
    blob = Blob(1.0, (0.25, 0.2, 0.2), (0.0, 0.0, 0.0), (0.2, 0.1, 0.0))
    dt, H = 0.06, 72
    p = Problem("tiles", src, obs, None, dt, H, H, [], MovingGaussians([blob], noise=0.02, seed=4))
    hist = history(p)
    prm = jefi.default_params(dt=dt, history_slots=H, precision="fp32c", tile_shape=shape)
    h = jefi.jefi_create(jefi.grid_from(src), obs_grid=jefi.grid_from(obs), params=prm)
    push_all(h, hist)
    assert jefi.jefi_get_info(h)["tile_shape"] == shape
    _, hi = jefi.jefi_valid_window(h)
    ref = oracle_fields(p, hist, [hi])
    E, B = gpu_fields(h, [hi])
    assert rel_l2(E[0], ref[0][0]) <= FP32C_TOL and rel_l2(B[0], ref[0][1]) <= FP32C_TOL
    got = jefi.jefi_debug_slots(h, hi)
    want = oracle.all_slots(src.n, src.lo, src.d, obs.points(), dt=dt, t0=0.0, c=1.0, t=hi)
    scr = want == oracle.SCREENED
    assert np.array_equal(got[~scr].astype(np.int64), want[~scr])
    assert jefi.jefi_get_info(h)["device_status"] == 0
    jefi.jefi_destroy(h)
    auto = jefi.jefi_create(jefi.grid_from(src), obs_grid=jefi.grid_from(obs),
                            params=jefi.default_params(dt=dt, history_slots=H, precision="fp32c"))
    assert jefi.jefi_get_info(auto)["tile_shape"] in range(1, 10)
    jefi.jefi_destroy(auto)
