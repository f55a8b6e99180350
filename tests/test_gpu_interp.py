"""GPU parity of the second-order retarded time (JEFI_FLAG_INTERP) against
the oracle's interpolated sum, through the C ABI.

Tolerances as for the floor rule: FP64 rel-L2 <= 1e-12, compensated FP32
rel-L2 <= 1e-5, normwise per field over all points and times.
"""
import numpy as np
import pytest

import oracle
import paper_2104_05426_gb300 as jefi
from jefi_cases import create, gpu_fields, history, push_all, rel_l2
from workloads import Blob, Dipole, Grid, MovingGaussians, Problem, c1_lienard_wiechert, shell_points

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32C_TOL = 1e-5
INTERP = jefi.JEFI_FLAG_INTERP


def oracle_interp(p, hist, times, supplied):
    rho, J, drho, dJ = hist
    kw = dict(drho=drho, dJ=dJ) if supplied else {}
    return [oracle.fields_interp(p.src.n, p.src.lo, p.src.d, p.obs(), rho, J, c=p.c, k_e=p.k_e,
                                 k_b=p.k_b, dt=p.dt, t0=p.t0, t=t, **kw) for t in times]


def check(h, p, hist, times, supplied, tol, tag=""):
    ref = oracle_interp(p, hist, times, supplied)
    E, B = gpu_fields(h, times)
    for i in range(len(times)):
        assert rel_l2(E[i], ref[i][0]) <= tol, (tag, i, rel_l2(E[i], ref[i][0]))
        assert rel_l2(B[i], ref[i][1]) <= tol, (tag, i, rel_l2(B[i], ref[i][1]))
    assert jefi.jefi_get_info(h)["device_status"] == 0


@pytest.fixture(scope="module")
def c1():
    p = c1_lienard_wiechert()
    return p, history(p)


def dipole_case():
    """Supplied derivatives (analytic), explicit points, c != 1, k_e != k_b."""
    src = Grid.cube(12, -0.5, 0.5)
    pts = shell_points([3.0, 6.0], 300, seed=5)
    c, dt, H = 2.0, 0.05, 96
    t0 = -(6.9 / c + 2 * dt)
    p = Problem("dip", src, None, pts, dt, H, H, [], Dipole(1.0, 2 * np.pi / 8.0, 0.1), c=c, k_e=0.7,
                k_b=0.7 / c ** 2, t0=t0)
    return p, history(p)


@pytest.fixture(scope="module")
def cases(c1):
    return {False: c1, True: dipole_case()}


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32c", FP32C_TOL)])
@pytest.mark.parametrize("supplied", [False, True])
def test_interp_matches_oracle(gpu, cases, prec, tol, supplied):
    """Central differences (C1, moving charge) and supplied derivatives
    (Hertz dipole)."""
    p, hist = cases[supplied]
    h = create(p, prec, supplied=supplied, flags=INTERP)
    push_all(h, hist, supplied=supplied)
    lo, hi = jefi.jefi_valid_window(h)
    times = [hi - 0.37, hi - 0.2, hi - 0.013, hi]
    check(h, p, hist, times, supplied, tol, (prec, supplied))
    if prec != "fp64":
        # both take the staged kernel: C1's lattice tiles by their boxes, the
        # dipole's shell points (radial tile order) by their distance shells
        assert jefi.jefi_get_info(h)["staged_band"] > 0
    jefi.jefi_destroy(h)


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32c", FP32C_TOL)])
def test_interp_non_lattice_ragged_grid(gpu, prec, tol):
    """Ragged, non-dyadic grids (padding cells, non-exact FP32 geometry with
    FP64 fall-backs) and observation points on and between source cells
    (screened and near pairs)."""
    src = Grid((13, 10, 7), (-0.731, -0.683, -0.402), (0.0931, 0.1377, 0.1013))
    rng = np.random.Generator(np.random.PCG64(21))
    near = src.points()[rng.choice(src.size, 300, replace=False)] + rng.uniform(-0.03, 0.03, (300, 3))
    far = rng.uniform(-2.5, 2.5, (700, 3))
    obs = np.concatenate([near, far])
    blob = Blob(0.8, (0.25, 0.3, 0.2), (-0.1, 0.05, 0.0), (0.3, -0.2, 0.1))
    dt, H = 0.0617, 120
    p = Problem("ragged", src, None, obs, dt, H, H, [], MovingGaussians([blob], noise=0.02, seed=4))
    hist = history(p)
    h = create(p, prec, flags=INTERP)
    push_all(h, hist)
    lo, hi = jefi.jefi_valid_window(h)
    check(h, p, hist, [hi - 0.5, hi - 0.11, hi], False, tol, prec)
    jefi.jefi_destroy(h)


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32c", FP32C_TOL)])
def test_interp_ring_wrap_and_window_edges(gpu, prec, tol):
    """A ring of 40 slices after 130 pushes: slots and their central
    differences wrap around the ring (and its mirror rows); times at both
    ends of the valid window."""
    src = Grid.cube(8, -0.5, 0.5)
    obs = Grid.box((8, 8, 8), (1.0, -0.5, -0.5), (2.0, 0.5, 0.5))
    blob = Blob(1.0, (0.15, 0.15, 0.15), (-0.2, 0.0, 0.0), (0.25, 0.0, 0.05))
    dt, H, n_push = 0.0625, 40, 130
    p = Problem("wrap", src, obs, None, dt, H, n_push, [], MovingGaussians([blob], noise=0.02, seed=5))
    hist = history(p)
    h = create(p, prec, H=H, flags=INTERP)
    push_all(h, hist)
    lo, hi = jefi.jefi_valid_window(h)
    assert np.isfinite(lo) and lo < hi
    check(h, p, hist, [lo, lo + 0.003, 0.5 * (lo + hi), hi - 0.004, hi], False, tol, prec)
    jefi.jefi_destroy(h)


@pytest.mark.parametrize("supplied", [False, True])
def test_interp_valid_window_ends_one_or_two_slices_early(gpu, cases, supplied):
    """Interpolation reads slice n+1 (and n+2 through a central difference):
    the window's upper end moves back by dt (2 dt); just past it the call
    refuses with ENOTYET and writes nothing."""
    p, hist = cases[supplied]
    h_floor = create(p, "fp64", supplied=supplied)
    h = create(p, "fp64", supplied=supplied, flags=INTERP)
    for x in (h_floor, h):
        push_all(x, hist, supplied=supplied)
    _, hi_floor = jefi.jefi_valid_window(h_floor)
    _, hi = jefi.jefi_valid_window(h)
    ahead = 1 if supplied else 2
    assert abs((hi_floor - hi) - ahead * p.dt) < 1e-9 * max(1.0, abs(hi))
    jefi.eval_fields(h, hi)
    with pytest.raises(jefi.JefiError) as e:
        jefi.eval_fields(h, hi + 1e-9 * max(1.0, abs(hi)))
    assert e.value.code == jefi.JEFI_ENOTYET
    for x in (h_floor, h):
        jefi.jefi_destroy(x)


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32c", FP32C_TOL)])
def test_interp_causal_start(gpu, prec, tol):
    """Times at which pairs retard into slices -1 and 0: zero history before
    the first slice, f'[0] = f[1] / (2 dt)."""
    src = Grid.cube(8, -0.5, 0.5)
    obs = Grid.box((8, 8, 4), (0.8, -0.5, -0.25), (1.6, 0.5, 0.25))
    blob = Blob(1.0, (0.2, 0.2, 0.2), (0.0, 0.0, 0.0), (0.1, 0.0, 0.0))
    dt, H = 0.05, 64
    p = Problem("start", src, obs, None, dt, H, H, [], MovingGaussians([blob], noise=0.05, seed=6))
    hist = history(p)
    h = create(p, prec, flags=INTERP)
    push_all(h, hist)
    check(h, p, hist, [0.3, 0.85, 1.05, 1.4], False, tol, prec)
    jefi.jefi_destroy(h)


def test_interp_second_order_through_the_library(gpu):
    """One cell with charge sin(omega t): against the closed-form retarded
    Coulomb + drho/(c R^2) field the interpolated sum is far more accurate
    than the floor rule at the same dt (FP64 and compensated FP32)."""
    src = Grid((1, 1, 1), (-0.05, -0.05, -0.05), (0.1, 0.1, 0.1))
    rng = np.random.Generator(np.random.PCG64(11))
    v = rng.standard_normal((64, 3))
    obs = v / np.linalg.norm(v, axis=1, keepdims=True) * rng.uniform(1.5, 3.0, 64)[:, None]
    om, dt, t = 2.0, 0.08, 6.0
    n_sl = int(t / dt) + 4
    rho = np.sin(om * dt * np.arange(n_sl))[:, None]
    J = np.zeros((n_sl, 1, 3))
    R = np.linalg.norm(obs, axis=1)
    tr = t - R
    E_ex = 1e-3 * obs * (np.sin(om * tr) / R**3 + om * np.cos(om * tr) / R**2)[:, None]
    errs = {}
    for prec in ("fp64", "fp32c"):
        for flags in (0, INTERP):
            prm = jefi.default_params(dt=dt, history_slots=n_sl, precision=prec, flags=flags)
            h = jefi.jefi_create(jefi.grid_from(src), obs_points=obs, params=prm)
            for n in range(n_sl):
                jefi.jefi_push_sources(h, rho[n], J[n])
            E, _ = jefi.eval_fields(h, t)
            errs[(prec, flags)] = rel_l2(E.cpu().numpy(), E_ex)
            jefi.jefi_destroy(h)
    for prec in ("fp64", "fp32c"):
        assert errs[(prec, INTERP)] < 0.05 * errs[(prec, 0)], errs


@pytest.mark.parametrize("lattice", [True, False])
def test_interp_staged_and_direct_kernels_agree(gpu, lattice):
    """The staged and the direct-gather FP32 kernels interpolate the same
    rows with the same weights: fields equal to FP32 rounding, both within
    tolerance of the oracle."""
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
    p = Problem("sd", src, obs, None, dt, H, H, [], MovingGaussians([blob], noise=0.02, seed=3))
    hist = history(p)
    hs = {name: create(p, "fp32c", flags=INTERP | extra)
          for name, extra in (("staged", 0), ("direct", jefi.JEFI_FLAG_DIRECT_GATHER))}
    for h in hs.values():
        push_all(h, hist)
    assert jefi.jefi_get_info(hs["staged"])["staged_band"] > 0
    assert jefi.jefi_get_info(hs["direct"])["staged_band"] == 0
    _, hi = jefi.jefi_valid_window(hs["staged"])
    times = [hi - 0.4, hi - 0.02]
    ref = oracle_interp(p, hist, times, False)
    out = {k: gpu_fields(h, times) for k, h in hs.items()}
    for i in range(len(times)):
        for k in out:
            assert rel_l2(out[k][0][i], ref[i][0]) <= FP32C_TOL
            assert rel_l2(out[k][1][i], ref[i][1]) <= FP32C_TOL
        assert rel_l2(out["staged"][0][i], out["direct"][0][i]) <= 2e-6
        assert rel_l2(out["staged"][1][i], out["direct"][1][i]) <= 2e-6
    for h in hs.values():
        jefi.jefi_destroy(h)


@pytest.mark.parametrize("prec,tol", [("fp64", FP64_TOL), ("fp32c", FP32C_TOL)])
def test_interp_in_batched_launch(gpu, c1, cases, prec, tol):
    """The batched kernels run the second-order rule for the handles that ask
    for it, beside floor-rule handles in the same batch: each result is
    bit-identical to its single evaluation and within tolerance of the
    oracle's second-order sum (staged kernel: C1 lattice; direct gather: the
    same problem forced onto it; the dipole's supplied derivatives)."""
    import torch

    p, hist = c1
    pd, hd = cases[True]
    hs = [create(p, prec, flags=INTERP), create(p, prec, flags=INTERP | jefi.JEFI_FLAG_DIRECT_GATHER),
          create(p, prec), create(pd, prec, supplied=True, flags=INTERP)]
    for h in hs[:3]:
        push_all(h, hist)
    push_all(hs[3], hd, supplied=True)
    ts = []
    for h in hs:
        lo, hi = jefi.jefi_valid_window(h)
        ts.append(hi - 0.13)
    Es = [torch.full((h.n_obs, 3), 7.0, dtype=torch.float64, device="cuda") for h in hs]
    Bs = [torch.full_like(E, 7.0) for E in Es]
    jefi.jefi_eval_batch(hs, ts, Es, Bs)
    torch.cuda.synchronize()
    for i, h in enumerate(hs):
        E1, B1 = jefi.eval_fields(h, ts[i])
        assert torch.equal(E1, Es[i]) and torch.equal(B1, Bs[i]), i
    for i, (prob, hh, sup) in enumerate(((p, hist, False), (p, hist, False), (pd, hd, True))):
        k = (0, 1, 3)[i]
        rho, J, drho, dJ = hh
        kw = dict(drho=drho, dJ=dJ) if sup else {}
        Er, Br = oracle.fields_interp(prob.src.n, prob.src.lo, prob.src.d, prob.obs(), rho, J, c=prob.c,
                                      k_e=prob.k_e, k_b=prob.k_b, dt=prob.dt, t0=prob.t0, t=ts[k], **kw)
        assert rel_l2(Es[k].cpu().numpy(), Er) <= tol and rel_l2(Bs[k].cpu().numpy(), Br) <= tol
    for h in hs:
        assert jefi.jefi_get_info(h)["device_status"] == 0
        jefi.jefi_destroy(h)


def test_view_creation_keeps_the_base_central_difference_state(gpu, c1):
    """Creating a view in the middle of the pushes must not touch the base's
    difference state (the view shares it): the base then gives the same
    fields as a twin that never had a view."""
    import torch

    p, hist = c1
    n = hist[0].shape[0]
    a = create(p, "fp64", flags=INTERP)
    b = create(p, "fp64", flags=INTERP)
    push_all(a, hist, upto=n // 2)
    push_all(b, hist, upto=n // 2)
    view = jefi.jefi_create_view(a, obs_grid=jefi.grid_from(p.obs_grid))
    rho, J, _, _ = hist
    for k in range(n // 2, n):
        for h in (a, b):
            jefi.jefi_push_sources(h, torch.from_numpy(rho[k]).cuda(), torch.from_numpy(J[k]).cuda())
    _, hi = jefi.jefi_valid_window(b)
    Ea, Ba = jefi.eval_fields(a, [hi - 0.2, hi])
    Eb, Bb = jefi.eval_fields(b, [hi - 0.2, hi])
    assert torch.equal(Ea, Eb) and torch.equal(Ba, Bb)
    jefi.jefi_destroy(view)
    for h in (a, b):
        jefi.jefi_destroy(h)
