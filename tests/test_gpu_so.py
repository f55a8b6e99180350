"""S-O decomposition on one GPU (paper Sec. 2.2, Fig. 2): every pair of a
source box and an observation chunk evaluated by its own handle, the fields
of a chunk summed in box order by jefi_sum_fields.  Source boxes keep the
whole grid's lattice (jefi_params.src_origin) and push their region of the
whole grid's slices, so every pair's retarded slot is the whole problem's
(bit for bit) and the fields agree to the precision's rounding."""
import numpy as np
import pytest

import oracle
import paper_2104_05426_gb300 as jefi
from paper_2104_05426_gb300.decomp import SODecomposition
from workloads import Blob, Grid, MovingGaussians

pytestmark = pytest.mark.gpu


def _problem():
    # ragged, non-dyadic source grid with padding cells; observers overlap it (screening)
    src = Grid((13, 10, 9), (-0.61, -0.47, -0.42), (0.093, 0.101, 0.097))
    rng = np.random.Generator(np.random.PCG64(21))
    obs = rng.uniform(-1.2, 1.2, (900, 3))
    dt, H = 0.061, 72
    m = MovingGaussians([Blob(1.0, (0.2, 0.25, 0.22), (-0.1, 0.0, 0.05), (0.25, -0.1, 0.1))], noise=0.02, seed=5)
    rho, J, _, _ = m.history(src, H, dt)
    return src, obs, dt, H, rho, J


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32c", 1e-5)])
@pytest.mark.parametrize("src_parts,obs_parts", [((2, 1, 1), 1), ((2, 2, 1), 1), ((1, 1, 1), 3), ((2, 1, 2), 2)])
def test_pairs_sum_to_the_whole_problem(gpu, prec, tol, src_parts, obs_parts):
    import torch

    src, obs, dt, H, rho, J = _problem()
    g = jefi.grid_from(src)
    prm = dict(dt=dt, history_slots=H, precision=prec)
    whole = jefi.jefi_create(g, obs_points=obs, params=jefi.default_params(**prm))
    so = SODecomposition(g, obs, prm, src_parts=src_parts, obs_parts=obs_parts)
    for n in range(H):
        jefi.jefi_push_sources(whole, rho[n], J[n])
        so.push(torch.from_numpy(rho[n]).cuda(), torch.from_numpy(J[n]).cuda())
    lo, hi = jefi.jefi_valid_window(whole)
    for t in (hi - 0.2, hi):
        Ew, Bw = (x.cpu().numpy() for x in jefi.eval_fields(whole, t))
        E, B = (x.cpu().numpy() for x in so.fields(t))
        Er, Br = oracle.fields(src.n, src.lo, src.d, obs, rho, J, dt=dt, t=t)
        assert _rel(E, Er) <= tol and _rel(B, Br) <= tol
        # the pairs' slots are the whole problem's, pair by pair
        slots_w = jefi.jefi_debug_slots(whole, t)
        for p, h in so.handles.items():
            o, k = so.pairs[p]
            sub, org = so.boxes[k]
            b0, b1 = so.chunks[o]
            if b1 == b0 or sub.n[0] * sub.n[1] * sub.n[2] == 0:
                continue
            iz, iy, ix = np.meshgrid(np.arange(sub.n[2]) + org[2], np.arange(sub.n[1]) + org[1],
                                     np.arange(sub.n[0]) + org[0], indexing="ij")
            cols = ((iz * src.n[1] + iy) * src.n[0] + ix).reshape(-1)
            assert np.array_equal(jefi.jefi_debug_slots(h, t), slots_w[b0:b1][:, cols])
    for h in so.handles.values():
        assert jefi.jefi_get_info(h)["device_status"] == 0
    so.close()
    jefi.jefi_destroy(whole)


def test_region_push_from_host_arrays(gpu):
    """A source box pushed from host arrays of the whole grid holds the same
    history as one pushed from device arrays (fields bit-identical)."""
    import torch

    src, obs, dt, H, rho, J = _problem()
    g = jefi.grid_from(src)
    prm = dict(dt=dt, history_slots=H, precision="fp64")
    a = SODecomposition(g, obs, prm, src_parts=(2, 1, 1))
    b = SODecomposition(g, obs, prm, src_parts=(2, 1, 1))
    for n in range(H):
        a.push(rho[n], J[n])
        b.push(torch.from_numpy(rho[n]).cuda(), torch.from_numpy(J[n]).cuda())
    lo, hi = a.valid_window()
    assert lo <= hi
    Ea, Ba = a.fields(hi)
    Eb, Bb = b.fields(hi)
    assert torch.equal(Ea, Eb) and torch.equal(Ba, Bb)
    with pytest.raises(ValueError):
        jefi.jefi_push_sources_region(next(iter(a.handles.values())), rho[0][:-1], J[0], src.n, (0, 0, 0))
    a.close()
    b.close()
