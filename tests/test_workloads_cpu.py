"""The seeded workload generators produce the configurations the benchmarks
and tests are quoted on (CPU): grid sizes and extents, time steps, history
lengths, source parameters, and evaluation times whose every retarded slot
(Eq. tr-1, decided by the oracle's exact rule) lies in [1, n_push - 1], so
each time is inside the window of a ring holding the pushed slices."""
import math

import numpy as np
import pytest

import oracle
from workloads import c1_lienard_wiechert, c2_heavy_ion, c3_dipole, c4_batch, distance_range


def _extreme_slots(p, t):
    """Slots of the nearest and farthest (observation, source) centre pairs:
    the slot is monotone in the distance, so these bound every pair's."""
    obs = p.obs()
    src = p.src
    lo = np.array([src.lo[a] + 0.5 * src.d[a] for a in range(3)])
    hi = np.array([src.lo[a] + (src.n[a] - 0.5) * src.d[a] for a in range(3)])
    # nearest source centre per point (on the lattice), farthest corner centre
    idx = np.clip(np.round((obs - lo) / np.asarray(src.d)), 0, np.asarray(src.n) - 1)
    near = lo + idx * np.asarray(src.d)
    far = np.where(np.abs(obs - lo) > np.abs(obs - hi), lo, hi)
    d = np.asarray(src.d)
    screened = np.all(np.abs(obs - near) <= 0.5 * d, axis=1)
    # a screened nearest pair is not evaluated: its point's nearest evaluated
    # pair is a face neighbour of that cell (one cell along some axis)
    best = near.copy()
    if screened.any():
        cand = []
        for a in range(3):
            for sgn in (-1.0, 1.0):
                q = near[screened].copy()
                q[:, a] += sgn * d[a]
                inside = (q[:, a] >= lo[a] - 1e-12) & (q[:, a] <= hi[a] + 1e-12)
                r = np.where(inside, np.linalg.norm(obs[screened] - q, axis=1), np.inf)
                cand.append((r, q))
        rs = np.stack([c[0] for c in cand])
        k = np.argmin(rs, axis=0)
        best[screened] = np.stack([cand[j][1][i] for i, j in enumerate(k)])
    s_far = oracle.pair_slots(obs, far, t=t, t0=p.t0, c=p.c, dt=p.dt)
    s_near = oracle.pair_slots(obs, best, t=t, t0=p.t0, c=p.c, dt=p.dt)
    return int(s_far.min()), int(s_near.max())


def _assert_window(p):
    for t in p.times:
        lo_slot, hi_slot = _extreme_slots(p, t)
        assert lo_slot >= 1, (p.name, t, lo_slot)
        assert hi_slot <= p.n_push - 1, (p.name, t, hi_slot)


def test_c1_moving_charge_config():
    p = c1_lienard_wiechert()
    assert p.src.n == (16, 16, 16) and p.src.lo == (-1.0, -1.0, -1.0) and p.src.d[0] == 0.125
    assert p.obs_grid.n == (16, 16, 16) and p.obs_grid.lo == (2.0, -1.0, -1.0)
    assert p.dt == 0.0625 and p.H == 80 and p.n_push == 80 and len(p.times) == 4
    (b,) = p.source.blobs
    assert b.q == 1.0 and b.sigma == (0.2, 0.2, 0.2) and b.v == (0.3, 0.0, 0.0)
    rmin, rmax = distance_range(p.src, p.obs())
    assert math.isclose(rmin, 1.125) and math.isclose(rmax, math.sqrt(4.875 ** 2 + 2 * 1.875 ** 2))
    # 64 slices cannot hold one evaluation: the span of retarded slots exceeds 64
    assert (rmax - rmin) / p.dt + 2 > 64
    _assert_window(p)


def test_c2_heavy_ion_config():
    p = c2_heavy_ion()
    assert p.src.n == (64, 64, 64) and p.obs_grid.n == (64, 64, 64)
    assert p.src.lo == (-5.0, -5.0, -5.0) and p.src.d[0] == 10.0 / 64 and p.dt == p.src.d[0]
    assert p.H == 128 and p.n_push == 128 and len(p.times) == 8
    b1, b2 = p.source.blobs
    gamma = 1.0 / math.sqrt(1.0 - 0.995 ** 2)
    assert abs(gamma - 10.0) < 0.02
    for b, sgn in ((b1, 1.0), (b2, -1.0)):
        assert b.sigma[:2] == (1.0, 1.0) and math.isclose(b.sigma[2], 1.0 / gamma)
        assert b.v == (0.0, 0.0, sgn * 0.995)
        assert math.isclose(b.x0[2] + b.v[2] * 10.0, 0.0, abs_tol=1e-12)   # they meet at t = 10
    assert p.source.noise == 0.01
    _assert_window(p)


def test_c3_dipole_config():
    p = c3_dipole()
    assert p.src.n == (32, 32, 32) and p.src.lo == (-0.5, -0.5, -0.5)
    assert p.H == 256 and p.dt == 0.15625 and len(p.times) == 4
    r = np.linalg.norm(p.obs_points, axis=1)
    for R in (5.0, 10.0, 20.0, 40.0):
        assert np.sum(np.abs(r - R) < 1e-12 * R) == 1024
    assert p.source.omega == 2 * math.pi / 8 and p.source.sigma == 0.1
    _assert_window(p)


@pytest.mark.parametrize("seed", [4, 8])
def test_c4_batch_config(seed):
    probs = c4_batch(n_problems=64, seed=seed)
    sides = [p.src.n[0] for p in probs]
    osides = [p.obs_grid.n[0] for p in probs]
    Hs = [p.H for p in probs]
    assert 8 <= min(sides) and max(sides) <= 48 and 8 <= min(osides) and max(osides) <= 32
    assert 32 <= min(Hs) and max(Hs) <= 128
    for p in probs:
        assert 1 <= len(p.source.blobs) <= 4 and len(p.times) == 1
        for b in p.source.blobs:
            assert np.linalg.norm(b.v) <= 0.9 + 1e-12 and 0.1 <= b.sigma[0] <= 0.4
        _assert_window(p)
