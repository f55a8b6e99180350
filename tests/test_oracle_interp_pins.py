"""Pins of the oracle's second-order variant (sources interpolated at the
retarded time, Eq. tr-1 without the floor; derivatives supplied or central
differences, both interpolated).

The expectations are the continuous retarded sum of Eqs. E-1/B-1 evaluated
with numpy from closed-form time dependences, the known error of linear
interpolation, a pure-Python brute force on a tiny grid, and the order of
convergence in dt.  None of them calls the oracle twice.
"""
import math

import numpy as np
import pytest

import oracle
from workloads import Grid

RNG = np.random.Generator(np.random.PCG64(77))


def continuous_fields(grid, obs, t, *, c, k_e, k_b, screen, rho_fn, drho_fn, J_fn, dJ_fn):
    """Eqs. E-1/B-1 with each cell's sources evaluated at its exact retarded
    time t - R/c (numpy, vectorised over cells)."""
    ctr = grid.points()
    dV = float(np.prod(grid.d))
    E = np.zeros((len(obs), 3))
    B = np.zeros((len(obs), 3))
    cells = np.arange(grid.size)
    for o, x in enumerate(obs):
        D = x[None, :] - ctr
        keep = ~np.all(np.abs(D) <= screen[None, :], axis=1)
        D = D[keep]
        cl = cells[keep]
        R = np.sqrt((D[:, 0] * D[:, 0] + D[:, 1] * D[:, 1]) + D[:, 2] * D[:, 2])
        tr = t - R / c
        rho, drho = rho_fn(tr, cl), drho_fn(tr, cl)
        J, dJ = J_fn(tr, cl), dJ_fn(tr, cl)
        te = D * (rho / R**3 + drho / (c * R**2))[:, None] - dJ / (c * c * R)[:, None]
        V = J / (R**3)[:, None] + dJ / (c * R**2)[:, None]
        E[o] = k_e * dV * te.sum(axis=0)
        B[o] = k_b * dV * np.cross(V, D).sum(axis=0)
    return E, B


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def sample_history(rho_fn, J_fn, t0, dt, n_slices, ns):
    cells = np.arange(ns)
    ts = t0 + dt * np.arange(n_slices)
    rho = np.stack([rho_fn(np.full(ns, tk), cells) for tk in ts])
    J = np.stack([J_fn(np.full(ns, tk), cells) for tk in ts])
    return rho, J


def far_obs(n, centre=(0.0, 0.0, 0.0), rmin=1.4, rmax=2.2, seed=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return np.asarray(centre) + v * rng.uniform(rmin, rmax, n)[:, None]


GRID = Grid((4, 3, 5), (-0.2, -0.15, -0.25), (0.1, 0.1, 0.1))
C, K_E, K_B, T0, DT, H = 1.3, 0.7, 0.45, 0.3, 0.07, 90


def linear_time_sources(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = GRID.size
    a, b = rng.uniform(-1, 1, ns), rng.uniform(-1, 1, ns)
    A, Bv = rng.uniform(-1, 1, (ns, 3)), rng.uniform(-1, 1, (ns, 3))
    return (lambda t, c: a[c] + b[c] * t, lambda t, c: b[c],
            lambda t, c: A[c] + Bv[c] * t[:, None], lambda t, c: Bv[c] + 0.0 * t[:, None])


def test_interp_exact_for_sources_linear_in_time():
    """Linear interpolation and central differences reproduce a linear time
    dependence exactly, so the variant equals the continuous retarded sum.
    Pins the interpolation weights (w vs 1 - w), the central difference,
    t0 and every term of Eqs. E-1/B-1."""
    rho_fn, drho_fn, J_fn, dJ_fn = linear_time_sources(1)
    rho, J = sample_history(rho_fn, J_fn, T0, DT, H, GRID.size)
    obs = far_obs(24)
    scr = np.asarray(GRID.d) / 2
    for t in (T0 + 4.1, T0 + 5.37):    # every pair: 1 <= n and n + 2 < H
        E, B = oracle.fields_interp(GRID.n, GRID.lo, GRID.d, obs, rho, J, c=C, k_e=K_E, k_b=K_B,
                                    dt=DT, t0=T0, t=t)
        Ec, Bc = continuous_fields(GRID, obs, t, c=C, k_e=K_E, k_b=K_B, screen=scr, rho_fn=rho_fn,
                                   drho_fn=drho_fn, J_fn=J_fn, dJ_fn=dJ_fn)
        assert rel_l2(E, Ec) <= 1e-11
        assert rel_l2(B, Bc) <= 1e-11


def test_interp_error_for_sources_quadratic_in_time():
    """For f = a + b t + q t^2 the interpolated central difference is exact
    (b + 2 q t_r) and linear interpolation is high by exactly q w (1 - w) dt^2,
    w the fractional slice position of the retarded time."""
    rng = np.random.Generator(np.random.PCG64(2))
    ns = GRID.size
    a, b, q = (rng.uniform(-1, 1, ns) for _ in range(3))
    A, Bv, Q = (rng.uniform(-1, 1, (ns, 3)) for _ in range(3))
    rho_fn = lambda t, c: a[c] + b[c] * t + q[c] * t * t
    J_fn = lambda t, c: A[c] + Bv[c] * t[:, None] + Q[c] * (t * t)[:, None]
    rho, J = sample_history(rho_fn, J_fn, T0, DT, H, ns)

    def frac(t):
        u = (t - T0) / DT
        return u - np.floor(u)

    def bump(t):
        w = frac(t)
        return w * (1 - w) * DT * DT

    obs = far_obs(16, seed=4)
    scr = np.asarray(GRID.d) / 2
    t = T0 + 4.6
    E, B = oracle.fields_interp(GRID.n, GRID.lo, GRID.d, obs, rho, J, c=C, k_e=K_E, k_b=K_B,
                                dt=DT, t0=T0, t=t)
    Ec, Bc = continuous_fields(
        GRID, obs, t, c=C, k_e=K_E, k_b=K_B, screen=scr,
        rho_fn=lambda tr, c: rho_fn(tr, c) + q[c] * bump(tr),
        drho_fn=lambda tr, c: b[c] + 2 * q[c] * tr,
        J_fn=lambda tr, c: J_fn(tr, c) + Q[c] * bump(tr)[:, None],
        dJ_fn=lambda tr, c: Bv[c] + 2 * Q[c] * tr[:, None])
    assert rel_l2(E, Ec) <= 1e-10
    assert rel_l2(B, Bc) <= 1e-10
    # the same data through the first-order rule is visibly worse
    Ef, Bf = oracle.fields(GRID.n, GRID.lo, GRID.d, obs, rho, J, c=C, k_e=K_E, k_b=K_B,
                           dt=DT, t0=T0, t=t)
    assert rel_l2(Ef, Ec) > 100 * rel_l2(E, Ec)


def test_interp_supplied_derivatives_are_interpolated():
    """Supplied derivatives are used as given (not differenced), interpolated
    like the values: with a supplied derivative linear in time (deliberately
    not the derivative of the values) the variant equals the continuous sum
    with that derivative."""
    rho_fn, _, J_fn, _ = linear_time_sources(5)
    rng = np.random.Generator(np.random.PCG64(6))
    ns = GRID.size
    g0, g1 = rng.uniform(-2, 2, ns), rng.uniform(-2, 2, ns)
    G0, G1 = rng.uniform(-2, 2, (ns, 3)), rng.uniform(-2, 2, (ns, 3))
    drho_fn = lambda t, c: g0[c] + g1[c] * t
    dJ_fn = lambda t, c: G0[c] + G1[c] * t[:, None]
    rho, J = sample_history(rho_fn, J_fn, T0, DT, H, ns)
    drho, dJ = sample_history(drho_fn, dJ_fn, T0, DT, H, ns)
    obs = far_obs(12, seed=8)
    scr = np.asarray(GRID.d) / 2
    t = T0 + 3.3
    E, B = oracle.fields_interp(GRID.n, GRID.lo, GRID.d, obs, rho, J, c=C, k_e=K_E, k_b=K_B,
                                dt=DT, t0=T0, t=t, drho=drho, dJ=dJ)
    Ec, Bc = continuous_fields(GRID, obs, t, c=C, k_e=K_E, k_b=K_B, screen=scr, rho_fn=rho_fn,
                               drho_fn=drho_fn, J_fn=J_fn, dJ_fn=dJ_fn)
    assert rel_l2(E, Ec) <= 1e-11
    assert rel_l2(B, Bc) <= 1e-11


def brute_interp(grid, obs, rho, J, drho, dJ, *, c, k_e, k_b, dt, t0, t):
    """Pure-Python statement of the variant on a tiny grid (math.fsum)."""
    nx, ny, nz = grid.n
    H = rho.shape[0]
    dV = grid.d[0] * grid.d[1] * grid.d[2]

    def f(arr, k, cell, comp=None):
        if k < 0:
            return 0.0
        return float(arr[k, cell] if comp is None else arr[k, cell, comp])

    def fdot(arr, darr, k, cell, comp=None):
        if k < 0:
            return 0.0
        if darr is not None:
            return f(darr, k, cell, comp)
        return (f(arr, k + 1, cell, comp) - f(arr, k - 1, cell, comp)) / (2 * dt)

    out = []
    for x in obs:
        terms_e = [[], [], []]
        terms_b = [[], [], []]
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    ctr = [grid.lo[0] + (i + 0.5) * grid.d[0], grid.lo[1] + (j + 0.5) * grid.d[1],
                           grid.lo[2] + (k + 0.5) * grid.d[2]]
                    D = [x[a] - ctr[a] for a in range(3)]
                    if all(abs(D[a]) <= grid.d[a] / 2 for a in range(3)):
                        continue
                    R = math.sqrt((D[0] * D[0] + D[1] * D[1]) + D[2] * D[2])
                    u = ((t - t0) - R / c) / dt
                    n = math.floor(u)
                    w = u - n
                    if n + 1 < 0:
                        continue
                    assert n + (1 if drho is not None else 2) < H
                    cell = (k * ny + j) * nx + i
                    lerp = lambda g0, g1: (1 - w) * g0 + w * g1
                    r = lerp(f(rho, n, cell), f(rho, n + 1, cell))
                    dr = lerp(fdot(rho, drho, n, cell), fdot(rho, drho, n + 1, cell))
                    Jv = [lerp(f(J, n, cell, a), f(J, n + 1, cell, a)) for a in range(3)]
                    dJv = [lerp(fdot(J, dJ, n, cell, a), fdot(J, dJ, n + 1, cell, a)) for a in range(3)]
                    for a in range(3):
                        terms_e[a].append(D[a] * (r / R**3 + dr / (c * R**2)) - dJv[a] / (c * c * R))
                    V = [Jv[a] / R**3 + dJv[a] / (c * R**2) for a in range(3)]
                    cr = [V[1] * D[2] - V[2] * D[1], V[2] * D[0] - V[0] * D[2], V[0] * D[1] - V[1] * D[0]]
                    for a in range(3):
                        terms_b[a].append(cr[a])
        out.append([k_e * dV * math.fsum(terms_e[a]) for a in range(3)] +
                   [k_b * dV * math.fsum(terms_b[a]) for a in range(3)])
    out = np.array(out)
    return out[:, :3], out[:, 3:]


@pytest.mark.parametrize("supplied", [False, True])
def test_interp_bruteforce_tiny_including_causal_start(supplied):
    """Tiny grid, random histories, times at which some pairs retard into
    slices -1 and 0: zero history before the first slice, f'[0] = f[1]/(2 dt)
    for central differences."""
    g = Grid((2, 2, 1), (0.0, 0.0, 0.0), (0.3, 0.25, 0.2))
    Hs = 7
    rng = np.random.Generator(np.random.PCG64(9 + supplied))
    rho = rng.uniform(-1, 1, (Hs, g.size))
    J = rng.uniform(-1, 1, (Hs, g.size, 3))
    drho = rng.uniform(-1, 1, (Hs, g.size)) if supplied else None
    dJ = rng.uniform(-1, 1, (Hs, g.size, 3)) if supplied else None
    obs = np.array([[0.9, 0.1, 0.05], [-0.5, 0.6, 0.3], [0.2, -0.7, -0.4]])
    for t in (0.75, 0.9, 1.17):
        E, B = oracle.fields_interp(g.n, g.lo, g.d, obs, rho, J, c=1.1, k_e=0.9, k_b=1.2, dt=0.2,
                                    t0=0.05, t=t, drho=drho, dJ=dJ)
        Eb, Bb = brute_interp(g, obs, rho, J, drho, dJ, c=1.1, k_e=0.9, k_b=1.2, dt=0.2, t0=0.05, t=t)
        assert np.allclose(E, Eb, rtol=1e-13, atol=1e-13 * np.abs(Eb).max())
        assert np.allclose(B, Bb, rtol=1e-13, atol=1e-13 * np.abs(Bb).max())


def test_interp_second_order_convergence_in_dt():
    """One cell with charge sin(omega t): the continuous field is known in
    closed form (Coulomb term plus the drho/(c R^2) term at t - R/c).  The
    variant's error falls ~4x when dt halves; the floor rule's ~2x."""
    g = Grid((1, 1, 1), (-0.05, -0.05, -0.05), (0.1, 0.1, 0.1))
    om, c = 2.0, 1.0
    obs = far_obs(8, rmin=1.5, rmax=3.0, seed=11)
    t = 6.0
    D = obs                                   # the cell centre is the origin
    R = np.linalg.norm(D, axis=1)
    tr = t - R / c
    dV = 1e-3
    E_ex = dV * D * (np.sin(om * tr) / R**3 + om * np.cos(om * tr) / (c * R**2))[:, None]
    errs = {}
    for dt in (0.08, 0.04):
        n_sl = int(t / dt) + 4
        ts = dt * np.arange(n_sl)
        rho = np.sin(om * ts)[:, None]
        J = np.zeros((n_sl, 1, 3))
        # sources start at t0 = 0 with rho(0) = 0; the history is long enough
        # that no pair sees the start
        Ei, _ = oracle.fields_interp(g.n, g.lo, g.d, obs, rho, J, c=c, dt=dt, t=t)
        Ef, _ = oracle.fields(g.n, g.lo, g.d, obs, rho, J, c=c, dt=dt, t=t)
        errs[dt] = (rel_l2(Ei, E_ex), rel_l2(Ef, E_ex))
    ratio_i = errs[0.08][0] / errs[0.04][0]
    ratio_f = errs[0.08][1] / errs[0.04][1]
    assert 3.3 < ratio_i < 4.8, errs
    assert 1.6 < ratio_f < 2.5, errs
    assert errs[0.04][0] < 0.1 * errs[0.04][1]


def test_interp_needs_one_or_two_slices_ahead():
    """Central differences read slice n+2, supplied derivatives only n+1:
    the same time is valid for one and too early for the other."""
    g = Grid((1, 1, 1), (-0.05, -0.05, -0.05), (0.1, 0.1, 0.1))
    obs = np.array([[1.0, 0.0, 0.0]])          # R = 1
    Hs = 10
    rho = np.ones((Hs, 1))
    J = np.zeros((Hs, 1, 3))
    t = 1.0 + 0.1 * 8 + 0.05                  # u = 8.5: n = 8, n + 1 = 9 = H - 1
    oracle.fields_interp(g.n, g.lo, g.d, obs, rho, J, dt=0.1, t=t, drho=rho, dJ=J)
    with pytest.raises(ValueError):
        oracle.fields_interp(g.n, g.lo, g.d, obs, rho, J, dt=0.1, t=t)
