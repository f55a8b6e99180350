"""Batched evaluation (jefi_eval_batch): many problems of uneven sizes in one
persistent launch per kernel variant.  Every problem's result must be
bit-identical to evaluating it alone, whatever else is in the batch, and
match the oracle within the parity tolerances."""
import numpy as np
import pytest

import oracle
import paper_2104_05426_gb300 as jefi
from jefi_cases import create, history, push_all, rel_l2
from workloads import c4_batch

pytestmark = pytest.mark.gpu


def _alloc(h):
    import torch

    E = torch.full((h.n_obs, 3), float("nan"), dtype=torch.float64, device="cuda")
    return E, torch.full_like(E, float("nan"))


@pytest.fixture(scope="module")
def batch_problems():
    probs = c4_batch(n_problems=18, seed=5, src_sides=(6, 20), obs_sides=(5, 14), H_range=(32, 64))
    hists = [history(p) for p in probs]
    return probs, hists


def test_batch_results_equal_single_evaluations(gpu, batch_problems):
    import torch

    probs, hists = batch_problems
    precs = ["fp32c", "fp32c", "fp64", "fp32"]
    handles = []
    for k, (p, hst) in enumerate(zip(probs, hists)):
        flags = jefi.JEFI_FLAG_DIRECT_GATHER if k % 5 == 4 else 0
        h = create(p, precs[k % len(precs)], flags=flags)
        push_all(h, hst)
        handles.append(h)
    times = [p.times[0] for p in probs]
    alone = []
    for h, t in zip(handles, times):
        E, B = _alloc(h)
        jefi.jefi_eval_fields(h, t, E, B)
        alone.append((E, B))
    # the mix: reversed order, one handle twice at two times
    order = list(reversed(range(len(handles)))) + [0]
    t_mix = [times[i] for i in order]
    t_mix[-1] = times[0] - 0.25 * probs[0].dt
    outs = [_alloc(handles[i]) for i in order]
    jefi.jefi_eval_batch([handles[i] for i in order], t_mix, [o[0] for o in outs], [o[1] for o in outs])
    torch.cuda.synchronize()
    for j, i in enumerate(order[:-1]):
        assert torch.equal(outs[j][0], alone[i][0]), i
        assert torch.equal(outs[j][1], alone[i][1]), i
    E2, B2 = _alloc(handles[0])
    jefi.jefi_eval_fields(handles[0], t_mix[-1], E2, B2)
    assert torch.equal(outs[-1][0], E2) and torch.equal(outs[-1][1], B2)
    # spot checks against the oracle
    for i in (0, 2, 5):
        p = probs[i]
        rho, J, _, _ = hists[i]
        Er, Br = oracle.fields(p.src.n, p.src.lo, p.src.d, p.obs(), rho, J, dt=p.dt, t0=p.t0, t=times[i])
        tol = 1e-12 if precs[i % len(precs)] == "fp64" else 1e-5
        assert rel_l2(alone[i][0].cpu().numpy(), Er) <= tol
        assert rel_l2(alone[i][1].cpu().numpy(), Br) <= tol
    for h in handles:
        assert jefi.jefi_get_info(h)["device_status"] == 0
        jefi.jefi_destroy(h)


def test_batch_rejects_bad_arguments(gpu, batch_problems):
    probs, hists = batch_problems
    h = create(probs[0], "fp32c")
    push_all(h, hists[0])
    E, B = _alloc(h)
    with pytest.raises(jefi.JefiError) as e:          # future slice
        jefi.jefi_eval_batch([h], [probs[0].times[0] + 50.0], [E], [B])
    assert e.value.code == jefi.JEFI_ENOTYET
    with pytest.raises(jefi.JefiError) as e:          # a handle more than 8 times
        jefi.jefi_eval_batch([h] * 9, [probs[0].times[0]] * 9, [E] * 9, [B] * 9)
    assert e.value.code == jefi.JEFI_EUNSUPPORTED
    jefi.jefi_destroy(h)


@pytest.mark.parametrize("direct", [False, True])
def test_fallback_count_single_equals_batched(gpu, direct):
    """Non-lattice geometry with many undecided pairs: the single-problem
    kernel counts its FP64 fall-backs per item in shared memory, the batched
    kernel per pair in global memory.  Both decide the same pairs, so the
    counts agree, and the fields are bit-identical.

    Source and observation centres differ by odd multiples of 1/60 on each
    axis, dt = sqrt(3)/20 and t is a whole number of steps: every pair on a
    body diagonal at a distance of a multiple of 3 * sqrt(3)/60 then sits on
    a slot boundary of Eq. tr-1, which FP32 cannot decide."""
    import torch

    from workloads import Blob, Grid, MovingGaussians, Problem

    src = Grid.box((12, 12, 12), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0))
    obs = Grid.box((20, 20, 20), (-2.0, -2.0, -2.0), (2.0, 2.0, 2.0))
    dt = float(np.sqrt(3.0)) / 20.0
    blob = Blob(1.0, (0.3, 0.25, 0.3), (-0.1, 0.05, 0.0), (0.2, 0.1, -0.05))
    prob = Problem("fb", src, obs, None, dt, 64, 64, [], MovingGaussians([blob], noise=0.02, seed=6))
    hist = history(prob)
    flags = jefi.JEFI_FLAG_DIRECT_GATHER if direct else 0
    h1, h2 = create(prob, "fp32c", flags=flags), create(prob, "fp32c", flags=flags)
    for h in (h1, h2):
        push_all(h, hist)
    assert (jefi.jefi_get_info(h1)["staged_band"] == 0) == direct
    lo, hi = jefi.jefi_valid_window(h1)
    t = prob.t0 + np.floor((hi - prob.t0) / dt) * dt
    assert lo <= t <= hi
    E1, B1 = _alloc(h1)
    jefi.jefi_eval_fields(h1, t, E1, B1)
    E2, B2 = _alloc(h2)
    jefi.jefi_eval_batch([h2], [t], [E2], [B2])
    torch.cuda.synchronize()
    n1 = jefi.jefi_get_info(h1)["slot_fallbacks"]
    n2 = jefi.jefi_get_info(h2)["slot_fallbacks"]
    assert n1 > 0 and n1 == n2
    assert torch.equal(E1, E2) and torch.equal(B1, B2)
    rho, J, _, _ = hist
    Er, Br = oracle.fields(src.n, src.lo, src.d, prob.obs(), rho, J, dt=dt, t0=prob.t0, t=t)
    assert rel_l2(E1.cpu().numpy(), Er) <= 1e-5 and rel_l2(B1.cpu().numpy(), Br) <= 1e-5
    for h in (h1, h2):
        assert jefi.jefi_get_info(h)["device_status"] == 0
        jefi.jefi_destroy(h)
