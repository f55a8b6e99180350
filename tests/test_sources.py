"""Self-tests of the seeded source generators (CPU): charge continuity.

Every source model feeding the oracle and the GPU path must satisfy
d rho/dt + div J = 0, as the paper notes for its sinusoidal sources
(Sec. 3.2); the moving Gaussians carry J = v rho and the dipole has
rho = -dP_z/dz, J = dP/dt.  Central differences on a fine grid give a
residual that is second order in the spacing and small against d rho/dt;
the dipole's supplied time derivatives must match differences in time."""
import math

import numpy as np
import pytest

from workloads import Blob, Dipole, Grid, MovingGaussians, OscBlob, OscillatingGaussians, Sinusoidal


def _residual(model, n, lo, hi, t, ht=1e-5):
    """Relative continuity residual on the interior cells, ||drho/dt + div J|| / ||drho/dt||."""
    g = Grid.cube(n, lo, hi)
    d = g.d[0]
    rho_p = model.sample(g, t + ht)[0]
    rho_m = model.sample(g, t - ht)[0]
    drho = ((rho_p - rho_m) / (2.0 * ht)).reshape(n, n, n)          # [z][y][x]
    J = model.sample(g, t)[1].reshape(n, n, n, 3)
    div = ((J[1:-1, 1:-1, 2:, 0] - J[1:-1, 1:-1, :-2, 0]) +
           (J[1:-1, 2:, 1:-1, 1] - J[1:-1, :-2, 1:-1, 1]) +
           (J[2:, 1:-1, 1:-1, 2] - J[:-2, 1:-1, 1:-1, 2])) / (2.0 * d)
    dr = drho[1:-1, 1:-1, 1:-1]
    return float(np.linalg.norm(dr + div) / np.linalg.norm(dr))


MODELS = {
    "sinusoidal (paper Sec. 3.2)": (Sinusoidal(), -3.0, 3.0, 2.3),
    "moving Gaussians": (MovingGaussians([Blob(1.0, (0.3, 0.25, 0.35), (0.1, -0.05, 0.0), (0.4, -0.2, 0.3)),
                                          Blob(-0.5, (0.2, 0.2, 0.2), (-0.2, 0.1, 0.1), (0.0, 0.5, -0.1))]),
                         -1.5, 1.5, 0.3),
    "dipole": (Dipole(1.0, 2.0 * math.pi / 8.0, 0.1), -0.5, 0.5, 1.1),
    "oscillating Gaussians": (OscillatingGaussians([OscBlob(1.0, (0.3, 0.25, 0.35), (0.1, -0.05, 0.0),
                                                            (0.2, -0.1, 0.15), 2.0, 0.3),
                                                    OscBlob(-0.5, (0.2, 0.2, 0.2), (-0.2, 0.1, 0.1),
                                                            (0.0, 0.25, -0.05), 1.3, 1.1)]),
                              -1.5, 1.5, 0.7),
}


@pytest.mark.parametrize("name", list(MODELS))
def test_sources_satisfy_continuity(name):
    model, lo, hi, t = MODELS[name]
    r1 = _residual(model, 40, lo, hi, t)
    r2 = _residual(model, 80, lo, hi, t)
    assert r2 < 2e-2, (r1, r2)
    assert r1 / r2 > 3.0, (r1, r2)        # second order in the spacing: the residual is the difference error


def test_dipole_supplied_derivatives_match_time_differences():
    model = Dipole(1.0, 2.0 * math.pi / 8.0, 0.1)
    g = Grid.cube(16, -0.5, 0.5)
    t, h = 1.7, 1e-5
    rho, J, drho, dJ = model.sample(g, t)
    rp, Jp, _, _ = model.sample(g, t + h)
    rm, Jm, _, _ = model.sample(g, t - h)
    assert np.allclose(drho, (rp - rm) / (2 * h), rtol=1e-6, atol=1e-9 * np.abs(drho).max())
    assert np.allclose(dJ, (Jp - Jm) / (2 * h), rtol=1e-6, atol=1e-9 * np.abs(dJ).max())


def test_device_form_of_moving_gaussians_matches_the_numpy_form():
    """The serving loop generates its slices with ``sample_torch`` (on the
    device); it is the same source model as ``sample`` (pinned above)."""
    import torch

    m = MovingGaussians([Blob(1.0, (0.2, 0.3, 0.25), (0.1, -0.2, 0.0), (0.3, 0.1, -0.2)),
                         Blob(-0.5, (0.3, 0.3, 0.3), (-0.2, 0.1, 0.2), (0.0, 0.4, 0.1))])
    g = Grid((7, 6, 5), (-1.0, -0.9, -0.8), (0.3, 0.31, 0.33))
    for t in (0.0, 0.7, 2.5):
        rho, J = m.sample(g, t)
        rt, Jt = m.sample_torch(torch.from_numpy(g.points()), t)
        assert np.allclose(rt.numpy(), rho, rtol=1e-13, atol=1e-13 * np.abs(rho).max())
        # components that cancel between blobs are compared at the field's scale
        # (numpy's and torch's exp may differ by an ulp, on some hosts)
        assert np.allclose(Jt.numpy(), J, rtol=1e-13, atol=1e-13 * np.abs(J).max())


def test_device_form_of_oscillating_gaussians_matches_the_numpy_form():
    import torch

    m = OscillatingGaussians([OscBlob(1.0, (0.2, 0.3, 0.25), (0.1, -0.2, 0.0), (0.3, 0.1, -0.2), 1.7, 0.4)])
    g = Grid((7, 6, 5), (-1.0, -0.9, -0.8), (0.3, 0.31, 0.33))
    for t in (0.0, 0.9, 31.5):
        rho, J = m.sample(g, t)
        rt, Jt = m.sample_torch(torch.from_numpy(g.points()), t)
        assert np.allclose(rt.numpy(), rho, rtol=1e-13, atol=1e-13 * np.abs(rho).max())
        # components that cancel between blobs are compared at the field's scale
        # (numpy's and torch's exp may differ by an ulp, on some hosts)
        assert np.allclose(Jt.numpy(), J, rtol=1e-13, atol=1e-13 * np.abs(J).max())


def test_batched_slices_of_many_problems_match_each_model():
    """The serving loop's batched slice generator (every problem's next slice
    in a few device operations per blob slot) gives each problem exactly what
    its own source model gives, blob counts differing between problems."""
    torch = pytest.importorskip("torch")
    from paper_2104_05426_gb300.serving import SliceBatch

    class Stub:
        def __init__(self, n, blobs):
            ax = torch.linspace(-1.0, 1.0, n, dtype=torch.float64)
            z, y, x = torch.meshgrid(ax, ax, ax, indexing="ij")
            self.pts = torch.stack([x.reshape(-1), y.reshape(-1), z.reshape(-1)], dim=1)
            self.blobs = blobs
            self.model = OscillatingGaussians(blobs)

    rng = np.random.Generator(np.random.PCG64(5))

    def blob():
        return OscBlob(float(rng.choice([-1.0, 1.0])), tuple(rng.uniform(0.15, 0.35, 3)),
                       tuple(rng.uniform(-0.2, 0.2, 3)), tuple(rng.uniform(-0.5, 0.5, 3)),
                       float(rng.uniform(0.5, 2.0)), float(rng.uniform(0.0, 6.0)))

    probs = [Stub(n, [blob() for _ in range(nb)]) for n, nb in ((5, 1), (7, 4), (4, 2), (6, 3))]
    sb = SliceBatch(probs)
    times = [0.0, 0.37, 1.9, 12.25]
    rho, J = sb.sample(times)
    for i, p in enumerate(probs):
        r_ref, j_ref = p.model.sample_torch(p.pts, times[i])
        a, b = int(sb.offsets[i]), int(sb.offsets[i + 1])
        assert torch.equal(rho[a:b], r_ref), i
        assert torch.equal(J[a:b], j_ref), i
