"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only *generates inputs*: grids, observation points and analytic
source densities rho(r, t), J(r, t) sampled at cell centres and slice times.
It contains none of the field-evaluation arithmetic; the oracle and the GPU
library each do that on their own.  Every random draw comes from
``numpy.random.Generator(PCG64(seed))``.

Source models (the paper's test sources and the heavier workloads built on
them):

* ``StepConstant``   rho = 1, J = (1, 1, 1) for t >= 0 (paper Sec. 3.1, Eq. const_sources)
* ``Sinusoidal``     rho = 3 (cos t - 1) cos(x+y+z), J_a = sin(x+y+z) sin t
                     for t >= 0 (paper Sec. 3.2, Eq. sin_sources)
* ``MovingGaussians`` sums of rigidly moving Gaussian charges, J = v rho,
                     with optional seeded uniform noise (heavy-ion-shaped)
* ``Dipole``         Gaussian-smeared oscillating dipole P = p(t) g(r) z-hat,
                     rho = -div P, J = dP/dt, with analytic time derivatives
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np


# --------------------------------------------------------------------------- grids
@dataclass(frozen=True)
class Grid:
    """Cell-centred grid: centre of cell i on axis a is lo[a] + (i + 0.5) d[a]."""

    n: Tuple[int, int, int]
    lo: Tuple[float, float, float]
    d: Tuple[float, float, float]

    @staticmethod
    def cube(side: int, lo: float, hi: float) -> "Grid":
        d = (hi - lo) / side
        return Grid((side,) * 3, (lo,) * 3, (d,) * 3)

    @staticmethod
    def box(n, lo, hi) -> "Grid":
        n = tuple(int(v) for v in n)
        lo = tuple(float(v) for v in lo)
        d = tuple((float(h) - float(l)) / k for l, h, k in zip(lo, hi, n))
        return Grid(n, lo, d)

    @property
    def size(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])

    @property
    def dV(self) -> float:
        return self.d[0] * self.d[1] * self.d[2]

    def axis(self, a: int) -> np.ndarray:
        return self.lo[a] + (np.arange(self.n[a], dtype=np.float64) + 0.5) * self.d[a]

    def points(self) -> np.ndarray:
        """All cell centres, [size, 3], x fastest."""
        z, y, x = np.meshgrid(self.axis(2), self.axis(1), self.axis(0), indexing="ij")
        return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def shell_points(radii: Sequence[float], per_shell: int, seed: int) -> np.ndarray:
    """Seeded points on spheres about the origin (directions from normalised Gaussians)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = []
    for r in radii:
        v = rng.standard_normal((per_shell, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        pts.append(r * v)
    return np.concatenate(pts, axis=0)


# --------------------------------------------------------------------------- sources
class SourceModel:
    """rho, J (and optionally their time derivatives) at cell centres at time t."""

    has_derivatives = False

    def sample(self, grid: Grid, t: float, slice_index: int = 0):
        raise NotImplementedError

    def history(self, grid: Grid, n_slices: int, dt: float, t0: float = 0.0):
        """Stacked slices n = 0 .. n_slices-1 at times t0 + n dt."""
        rho = np.empty((n_slices, grid.size))
        J = np.empty((n_slices, grid.size, 3))
        drho = np.empty((n_slices, grid.size)) if self.has_derivatives else None
        dJ = np.empty((n_slices, grid.size, 3)) if self.has_derivatives else None
        for n in range(n_slices):
            out = self.sample(grid, t0 + n * dt, n)
            rho[n], J[n] = out[0], out[1]
            if self.has_derivatives:
                drho[n], dJ[n] = out[2], out[3]
        return rho, J, drho, dJ


class StepConstant(SourceModel):
    def sample(self, grid, t, slice_index=0):
        on = 1.0 if t >= 0 else 0.0
        return np.full(grid.size, on), np.full((grid.size, 3), on)


class Sinusoidal(SourceModel):
    def sample(self, grid, t, slice_index=0):
        p = grid.points()
        s = p.sum(axis=1)
        if t < 0:
            return np.zeros(grid.size), np.zeros((grid.size, 3))
        rho = 3.0 * (math.cos(t) - 1.0) * np.cos(s)
        j = np.sin(s) * math.sin(t)
        return rho, np.repeat(j[:, None], 3, axis=1)


@dataclass
class Blob:
    q: float
    sigma: Tuple[float, float, float]
    x0: Tuple[float, float, float]      # centre at t = 0
    v: Tuple[float, float, float]


def gaussian3(p: np.ndarray, centre, sigma) -> np.ndarray:
    """Normalised anisotropic Gaussian density at points p."""
    s = np.asarray(sigma, dtype=np.float64)
    u = (p - np.asarray(centre, dtype=np.float64)) / s
    norm = 1.0 / ((2.0 * math.pi) ** 1.5 * s[0] * s[1] * s[2])
    return norm * np.exp(-0.5 * np.sum(u * u, axis=1))


@dataclass
class MovingGaussians(SourceModel):
    blobs: List[Blob]
    noise: float = 0.0          # relative amplitude of seeded uniform noise
    seed: int = 0
    _pts: dict = field(default_factory=dict, repr=False)
    _scale: Optional[float] = None

    def _points(self, grid):
        key = (grid.n, grid.lo, grid.d)
        if key not in self._pts:
            self._pts[key] = grid.points()
        return self._pts[key]

    def sample(self, grid, t, slice_index=0):
        p = self._points(grid)
        rho = np.zeros(grid.size)
        J = np.zeros((grid.size, 3))
        for b in self.blobs:
            c = np.asarray(b.x0) + np.asarray(b.v) * t
            g = b.q * gaussian3(p, c, b.sigma)
            rho += g
            J += g[:, None] * np.asarray(b.v)[None, :]
        if self.noise > 0.0:
            if self._scale is None:
                self._scale = max(abs(b.q) * float(gaussian3(np.zeros((1, 3)), (0, 0, 0), b.sigma)[0])
                                  for b in self.blobs)
            vmax = max(float(np.linalg.norm(b.v)) for b in self.blobs)
            rng = np.random.Generator(np.random.PCG64([self.seed, slice_index]))
            amp = self.noise * self._scale
            rho += rng.uniform(-amp, amp, grid.size)
            J += rng.uniform(-amp * vmax, amp * vmax, (grid.size, 3))
        return rho, J

    def sample_torch(self, pts, t):
        """The noise-free sample at time t for points ``pts`` ([N, 3] torch
        float64 tensor, any device), by the same formula as ``sample``: a
        slice generated where the points live (no host copy per slice)."""
        import torch

        rho = torch.zeros(pts.shape[0], dtype=pts.dtype, device=pts.device)
        J = torch.zeros((pts.shape[0], 3), dtype=pts.dtype, device=pts.device)
        for b in self.blobs:
            s = torch.tensor(b.sigma, dtype=pts.dtype, device=pts.device)
            c = torch.tensor([b.x0[a] + b.v[a] * t for a in range(3)], dtype=pts.dtype, device=pts.device)
            u = (pts - c) / s
            norm = 1.0 / ((2.0 * math.pi) ** 1.5 * b.sigma[0] * b.sigma[1] * b.sigma[2])
            g = (b.q * norm) * torch.exp(-0.5 * (u * u).sum(dim=1))
            rho += g
            J += g[:, None] * torch.tensor(b.v, dtype=pts.dtype, device=pts.device)[None, :]
        return rho, J


@dataclass
class OscBlob:
    """A Gaussian charge whose centre oscillates: c(t) = x0 + amp sin(omega t + phase)."""
    q: float
    sigma: Tuple[float, float, float]
    x0: Tuple[float, float, float]
    amp: Tuple[float, float, float]
    omega: float
    phase: float = 0.0


@dataclass
class OscillatingGaussians(SourceModel):
    """Rigidly moving Gaussian charges on bounded paths: rho = sum q G(r - c(t)),
    J = sum q G(r - c(t)) c'(t), which satisfies continuity like any rigid
    motion.  The charges stay near x0 forever, so a long-running history
    (the serving workload pushes a slice per tick) keeps its fields."""
    blobs: List[OscBlob]

    def _centre(self, b, t):
        s = math.sin(b.omega * t + b.phase)
        c = math.cos(b.omega * t + b.phase)
        return ([b.x0[a] + b.amp[a] * s for a in range(3)], [b.amp[a] * b.omega * c for a in range(3)])

    def sample(self, grid, t, slice_index=0):
        p = grid.points()
        rho = np.zeros(grid.size)
        J = np.zeros((grid.size, 3))
        for b in self.blobs:
            c, v = self._centre(b, t)
            g = b.q * gaussian3(p, c, b.sigma)
            rho += g
            J += g[:, None] * np.asarray(v)[None, :]
        return rho, J

    def sample_torch(self, pts, t):
        """The sample at time t for points ``pts`` ([N, 3] torch float64,
        any device), by the same formula as ``sample``."""
        import torch

        rho = torch.zeros(pts.shape[0], dtype=pts.dtype, device=pts.device)
        J = torch.zeros((pts.shape[0], 3), dtype=pts.dtype, device=pts.device)
        for b in self.blobs:
            c, v = self._centre(b, t)
            s = torch.tensor(b.sigma, dtype=pts.dtype, device=pts.device)
            u = (pts - torch.tensor(c, dtype=pts.dtype, device=pts.device)) / s
            norm = 1.0 / ((2.0 * math.pi) ** 1.5 * b.sigma[0] * b.sigma[1] * b.sigma[2])
            g = (b.q * norm) * torch.exp(-0.5 * (u * u).sum(dim=1))
            rho += g
            J += g[:, None] * torch.tensor(v, dtype=pts.dtype, device=pts.device)[None, :]
        return rho, J


@dataclass
class Dipole(SourceModel):
    """P(r, t) = p0 cos(omega t) g_sigma(r) z-hat; rho = -dP_z/dz, J = dP/dt."""

    p0: float
    omega: float
    sigma: float
    has_derivatives = True

    def sample(self, grid, t, slice_index=0):
        p = grid.points()
        g = gaussian3(p, (0.0, 0.0, 0.0), (self.sigma,) * 3)
        shape = p[:, 2] / (self.sigma ** 2) * g          # -d g / dz
        w = self.omega
        pt = self.p0 * math.cos(w * t)
        pd = -self.p0 * w * math.sin(w * t)
        pdd = -self.p0 * w * w * math.cos(w * t)
        rho = pt * shape
        drho = pd * shape
        J = np.zeros((grid.size, 3))
        dJ = np.zeros((grid.size, 3))
        J[:, 2] = pd * g
        dJ[:, 2] = pdd * g
        return rho, J, drho, dJ


# --------------------------------------------------------------------------- configs
@dataclass
class Problem:
    """One source/observation problem plus its history and evaluation times."""

    name: str
    src: Grid
    obs_grid: Optional[Grid]
    obs_points: Optional[np.ndarray]
    dt: float
    H: int
    n_push: int
    times: List[float]
    source: SourceModel
    c: float = 1.0
    k_e: float = 1.0
    k_b: float = 1.0
    t0: float = 0.0

    def obs(self) -> np.ndarray:
        return self.obs_grid.points() if self.obs_grid is not None else self.obs_points

    @property
    def n_obs(self) -> int:
        return self.obs_grid.size if self.obs_grid is not None else int(self.obs_points.shape[0])


def _eval_times(lo: float, hi: float, k: int) -> List[float]:
    if k == 1:
        return [0.5 * (lo + hi)]
    return [lo + (hi - lo) * (i + 0.5) / k for i in range(k)]


def distance_range(src: Grid, obs: np.ndarray) -> Tuple[float, float]:
    """Smallest and largest centre-to-centre distance (brute force over axes)."""
    lo = np.array([src.lo[a] + 0.5 * src.d[a] for a in range(3)])
    hi = np.array([src.lo[a] + (src.n[a] - 0.5) * src.d[a] for a in range(3)])
    near = np.clip(obs, lo, hi)
    rmin = float(np.min(np.linalg.norm(obs - near, axis=1)))
    far = np.where(np.abs(obs - lo) > np.abs(obs - hi), lo, hi)
    rmax = float(np.max(np.linalg.norm(obs - far, axis=1)))
    return rmin, rmax


def c1_lienard_wiechert(side: int = 16, H: int = 80, dt: float = 0.0625, n_times: int = 4) -> Problem:
    """Gaussian charge q = 1, sigma = 0.2 moving along +x at 0.3 c; sources
    16^3 over [-1,1]^3, observation 16^3 over [2,4] x [-1,1]^2; c = k = 1."""
    src = Grid.cube(side, -1.0, 1.0)
    obs = Grid.box((side,) * 3, (2.0, -1.0, -1.0), (4.0, 1.0, 1.0))
    rmin, rmax = distance_range(src, obs.points())
    n_push = H
    # valid window: every retarded slot >= 1 and <= n_push - 1
    t_lo = rmax + dt * 1.0001
    t_hi = (n_push - 1) * dt + rmin
    times = _eval_times(t_lo, min(t_hi, t_lo + 0.45), n_times)
    v = 0.3
    # charge centre crosses x = 0 when seen from the obs-grid centre (x=3) at the middle time
    tm = 0.5 * (times[0] + times[-1])
    tc = tm - 3.0  # retarded time of the centre distance 3 (c = 1)
    blob = Blob(1.0, (0.2, 0.2, 0.2), (-v * tc, 0.0, 0.0), (v, 0.0, 0.0))
    return Problem("C1", src, obs, None, dt, H, n_push, times, MovingGaussians([blob]))


def c2_heavy_ion(side: int = 64, H: int = 128, n_times: int = 8, noise: float = 0.01,
                 seed: int = 2) -> Problem:
    """Two Lorentz-contracted Gaussian blobs (sigma_T = 1, gamma = 10) at
    +-0.995 c along z colliding at t = 10, plus 1% seeded noise; both grids
    side^3 over [-5,5]^3, dt = cell size, c = k = 1."""
    src = Grid.cube(side, -5.0, 5.0)
    obs = Grid.cube(side, -5.0, 5.0)
    dt = src.d[0]
    v = 0.995
    gamma = 1.0 / math.sqrt(1.0 - v * v)
    sz = 1.0 / gamma
    t_coll = 10.0
    blobs = [Blob(1.0, (1.0, 1.0, sz), (0.0, 0.0, -v * t_coll), (0.0, 0.0, v)),
             Blob(1.0, (1.0, 1.0, sz), (0.0, 0.0, v * t_coll), (0.0, 0.0, -v))]
    rmax = math.sqrt(3.0) * 10.0
    n_push = H
    t_hi = (n_push - 1) * dt  # R_min (neighbour cells) ~ dt: keep slots <= n_push-1
    t_lo = t_hi - (H - 2) * dt + rmax
    times = _eval_times(max(t_lo, 0.0), t_hi, n_times)
    return Problem("C2", src, obs, None, dt, H, n_push, times,
                   MovingGaussians(blobs, noise=noise, seed=seed))


def c3_dipole(side: int = 32, per_shell: int = 1024, radii=(5.0, 10.0, 20.0, 40.0), H: int = 256,
              dt: float = 0.15625, n_times: int = 4, sigma: float = 0.1, seed: int = 3) -> Problem:
    """Gaussian-smeared dipole p0 cos(omega t), omega = 2 pi / 8, in 32^3 cells
    over [-0.5,0.5]^3; observation points on shells R = 5, 10, 20, 40."""
    src = Grid.cube(side, -0.5, 0.5)
    pts = shell_points(radii, per_shell, seed)
    rmin, rmax = distance_range(src, pts)
    span = (rmax - rmin) / dt
    t0 = -(rmax + 2 * dt)  # history starts early enough for the farthest pair
    n_push = H
    t_hi = t0 + (n_push - 1) * dt + rmin
    times = _eval_times(t_hi - 0.5, t_hi, n_times)
    assert span + 3 < H
    return Problem("C3", src, None, pts, dt, H, n_push, times,
                   Dipole(1.0, 2.0 * math.pi / 8.0, sigma), t0=t0)


def c4_batch(n_problems: int = 256, seed: int = 4, src_sides=(8, 48), obs_sides=(8, 32),
             H_range=(32, 128)) -> List[Problem]:
    """Independent problems of uneven sizes: cubic source grids of side
    uniform in src_sides over [-1,1]^3, cubic observation grids of side
    uniform in obs_sides over [-2,2]^3 (overlapping, so screening applies),
    1-4 moving Gaussian charges (speed uniform in [0, 0.9]c, random
    direction, sigma in [0.1, 0.4]), H uniform in H_range and
    dt = (R_max - R_min)/(c (H - 3)) so each history just covers its pairs;
    one evaluation time per problem, inside its window."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for k in range(n_problems):
        ns = int(rng.integers(src_sides[0], src_sides[1] + 1))
        no = int(rng.integers(obs_sides[0], obs_sides[1] + 1))
        H = int(rng.integers(H_range[0], H_range[1] + 1))
        src = Grid.cube(ns, -1.0, 1.0)
        obs = Grid.cube(no, -2.0, 2.0)
        blobs = []
        for _ in range(int(rng.integers(1, 5))):
            v = rng.standard_normal(3)
            v *= rng.uniform(0.0, 0.9) / np.linalg.norm(v)
            sig = float(rng.uniform(0.1, 0.4))
            x0 = rng.uniform(-0.3, 0.3, 3)
            blobs.append(Blob(float(rng.choice([-1.0, 1.0])), (sig, sig, sig), tuple(x0), tuple(v)))
        rmax = float(np.linalg.norm(np.array(obs.lo) - (np.array(src.lo) + np.array(src.d) * (np.array(src.n) - 0.5)))) + 1e-9
        rmin = min(src.d[0], obs.d[0]) * 0.25
        dt = (rmax - rmin) / (H - 3)
        # window: slots between 1 and H-1 for every pair; shift the charges so
        # they sit near the origin at the evaluation time
        t_eval = rmax + 1.5 * dt
        t0 = 0.0
        moved = [Blob(b.q, b.sigma, tuple(np.asarray(b.x0) - np.asarray(b.v) * (t_eval - 1.0)), b.v)
                 for b in blobs]
        out.append(Problem(f"C4-{k}", src, obs, None, dt, H, H, [t_eval], MovingGaussians(moved),
                           t0=t0))
    return out


def e1_constant(H: int = 256, n_push: int = 160) -> Problem:
    """Paper Sec. 3.1: step-on constant sources rho = 1, J = (1,1,1) for t >= 0;
    15^3 source and observation cells over [-3,3]^3 (cell 0.4), screening
    half-width 0.2 (half a cell), snapshots t = 2.5, 5, 7.5, dt = 0.05."""
    g = Grid.cube(15, -3.0, 3.0)
    return Problem("E1", g, g, None, 0.05, H, n_push, [2.5, 5.0, 7.5], StepConstant())


def e2_sinusoidal(H: int = 300, n_push: int = 200) -> Problem:
    """Paper Sec. 3.2: rho = 3(cos t - 1) cos(x+y+z), J_a = sin(x+y+z) sin t for
    t >= 0; sources 15^3 over [-3,3]^3, observers 15^3 over [-3,3]^2 x [10,16],
    dt = 0.05."""
    src = Grid.cube(15, -3.0, 3.0)
    obs = Grid.box((15, 15, 15), (-3.0, -3.0, 10.0), (3.0, 3.0, 16.0))
    return Problem("E2", src, obs, None, 0.05, H, n_push, [10.0, 12.5, 15.0], Sinusoidal())
