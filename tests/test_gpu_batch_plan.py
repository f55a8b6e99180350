"""Batch plans (jefi_batch_plan_*): a fixed batch recorded as CUDA graphs and
replayed at new times, and the autotuner of the batched launch.

A plan runs the batched kernels of jefi_eval_batch on the same handle
state, so every replay must be bit-identical to jefi_eval_batch at the same
times -- across launches, after further pushes, and after a handle's kernel
or split count changed (the plan records its graphs again).  The tuner
changes the handles' kernels and source splits: its results must stay within
the parity tolerances of the oracle."""
import numpy as np
import pytest

import oracle
import paper_2104_05426_gb300 as jefi
from jefi_cases import create, history, push_all, rel_l2
from workloads import c4_batch

pytestmark = pytest.mark.gpu

PRECS = ["fp32c", "fp64", "fp32c", "fp32"]


def _alloc(h):
    import torch

    E = torch.full((h.n_obs, 3), float("nan"), dtype=torch.float64, device="cuda")
    return E, torch.full_like(E, float("nan"))


@pytest.fixture(scope="module")
def plan_problems():
    probs = c4_batch(n_problems=10, seed=8, src_sides=(6, 20), obs_sides=(5, 14), H_range=(24, 64))
    hists = [history(p, p.n_push + 1) for p in probs]   # one slice beyond the first window
    return probs, hists


def _handles(probs, hists):
    hs = []
    for k, (p, hst) in enumerate(zip(probs, hists)):
        flags = jefi.JEFI_FLAG_DIRECT_GATHER if k % 5 == 4 else 0
        if k == 0:
            flags |= jefi.JEFI_FLAG_SHARED_RING
        h = create(p, PRECS[k % len(PRECS)], flags=flags)
        push_all(h, hst, upto=p.n_push)
        hs.append(h)
    view = jefi.jefi_create_view(hs[0], obs_grid=jefi.grid((7, 7, 7), (-1.5,) * 3, (3.0 / 7,) * 3))
    return hs, view


def _batch_reference(entries, ts):
    import torch

    outs = [_alloc(h) for h in entries]
    jefi.jefi_eval_batch(entries, ts, [o[0] for o in outs], [o[1] for o in outs])
    torch.cuda.synchronize()
    return outs


def _assert_equal(a, b):
    import torch

    for j, ((Ea, Ba), (Eb, Bb)) in enumerate(zip(a, b)):
        assert torch.equal(Ea, Eb) and torch.equal(Ba, Bb), j


def _check_oracle(probs, hists, k, E, B, t, n_slices):
    p = probs[k]
    rho, J, _, _ = hists[k]
    Er, Br = oracle.fields(p.src.n, p.src.lo, p.src.d, p.obs(), rho[:n_slices], J[:n_slices],
                           dt=p.dt, t0=p.t0, t=t)
    tol = 1e-12 if PRECS[k % len(PRECS)] == "fp64" else 1e-5
    assert rel_l2(E.cpu().numpy(), Er) <= tol, k
    assert rel_l2(B.cpu().numpy(), Br) <= tol, k


def test_plan_replays_equal_eval_batch(gpu, plan_problems):
    """Graph replays at new times and after a push equal jefi_eval_batch bit
    for bit; a handle twice (two times) and a view included."""
    import torch

    probs, hists = plan_problems
    hs, view = _handles(probs, hists)
    n = len(hs)
    entries = hs + [hs[0], view]
    outs = [_alloc(h) for h in entries]
    plan = jefi.jefi_batch_plan_create(entries, [o[0] for o in outs], [o[1] for o in outs])

    def times(shift):
        ts = [probs[i].times[0] + shift * probs[i].dt for i in range(n)]
        return ts + [probs[0].times[0], probs[0].times[0] + 0.5 * shift * probs[0].dt]

    for shift in (-0.25, 0.25, 0.0):
        ts = times(shift)
        jefi.jefi_batch_plan_launch(plan, ts)
        torch.cuda.synchronize()
        _assert_equal(outs, _batch_reference(entries, ts))
    # one more slice: the oldest is evicted, the window moves by dt
    for k in range(n):
        rho, J, _, _ = hists[k]
        jefi.jefi_push_sources(hs[k], torch.from_numpy(rho[probs[k].n_push]).cuda(),
                               torch.from_numpy(np.ascontiguousarray(J[probs[k].n_push])).cuda())
    ts = times(1.0)
    jefi.jefi_batch_plan_launch(plan, ts)
    torch.cuda.synchronize()
    _assert_equal(outs, _batch_reference(entries, ts))
    for k in (0, 1, 3):
        _check_oracle(probs, hists, k, outs[k][0], outs[k][1], ts[k], probs[k].n_push + 1)
    # a time outside a window: refused, nothing written
    for E, B in outs:
        E.fill_(float("nan"))
    bad = list(ts)
    bad[2] = ts[2] + 50.0
    with pytest.raises(jefi.JefiError) as e:
        jefi.jefi_batch_plan_launch(plan, bad)
    assert e.value.code == jefi.JEFI_ENOTYET
    torch.cuda.synchronize()
    assert all(bool(torch.isnan(E).all()) for E, _ in outs)
    # handles held by a live plan cannot be destroyed
    assert jefi.load().jefi_destroy(hs[1].ptr) == jefi.JEFI_EINVAL
    jefi.jefi_batch_plan_destroy(plan)
    for h in entries[-1:] + hs:
        assert jefi.jefi_get_info(h)["device_status"] == 0
        jefi.jefi_destroy(h)


def test_plan_records_again_after_kernel_switch(gpu, plan_problems):
    import torch

    probs, hists = plan_problems
    hs, view = _handles(probs, hists)
    entries = hs + [view]
    outs = [_alloc(h) for h in entries]
    plan = jefi.jefi_batch_plan_create(entries, [o[0] for o in outs], [o[1] for o in outs])
    ts = [p.times[0] for p in probs] + [probs[0].times[0]]
    staged = [k for k, h in enumerate(hs) if jefi.jefi_get_info(h)["staged_band"] > 0]
    assert staged
    for k in staged:
        jefi.jefi_select_kernel(hs[k], jefi.JEFI_KERNEL_DIRECT)
    jefi.jefi_batch_plan_launch(plan, ts)
    torch.cuda.synchronize()
    _assert_equal(outs, _batch_reference(entries, ts))
    for k in staged:
        assert jefi.jefi_get_info(hs[k])["staged_band"] == 0
        jefi.jefi_select_kernel(hs[k], jefi.JEFI_KERNEL_STAGED)
    jefi.jefi_batch_plan_launch(plan, ts)
    torch.cuda.synchronize()
    _assert_equal(outs, _batch_reference(entries, ts))
    _check_oracle(probs, hists, staged[0], outs[staged[0]][0], outs[staged[0]][1], ts[staged[0]],
                  probs[staged[0]].n_push)
    jefi.jefi_batch_plan_destroy(plan)
    for h in [view] + hs:
        jefi.jefi_destroy(h)


def test_tuner_keeps_parity(gpu, plan_problems):
    """The tuner times its candidates and leaves the fastest in the handles;
    tuned results match the oracle and jefi_eval_batch on the tuned handles."""
    import torch

    probs, hists = plan_problems
    hs, view = _handles(probs, hists)
    entries = hs + [view]
    splits0 = [jefi.jefi_get_info(h)["n_split"] for h in entries]
    outs = [_alloc(h) for h in entries]
    plan = jefi.jefi_batch_plan_create(entries, [o[0] for o in outs], [o[1] for o in outs])
    ts = [p.times[0] for p in probs] + [probs[0].times[0]]
    rep = jefi.jefi_batch_plan_tune(plan, ts)
    assert rep["candidates"] >= 2
    assert rep["split_divisor"] in (0, 1, 2, 4, 8)
    assert rep["measured_kernels"] in (0, 1) and rep["concurrent_groups"] in (0, 1)
    assert 0 < rep["ms_tuned"] <= rep["ms_initial"]
    for h, s0 in zip(entries, splits0):
        assert 1 <= jefi.jefi_get_info(h)["n_split"] <= s0
    for E, B in outs:
        E.fill_(float("nan"))
    jefi.jefi_batch_plan_launch(plan, ts)
    torch.cuda.synchronize()
    _assert_equal(outs, _batch_reference(entries, ts))
    for k in range(len(hs)):
        _check_oracle(probs, hists, k, outs[k][0], outs[k][1], ts[k], probs[k].n_push)
    # single evaluations use the tuned configuration too
    E1, B1 = _alloc(hs[0])
    jefi.jefi_eval_fields(hs[0], ts[0], E1, B1)
    torch.cuda.synchronize()
    assert torch.equal(E1, outs[0][0]) and torch.equal(B1, outs[0][1])
    jefi.jefi_batch_plan_destroy(plan)
    for h in [view] + hs:
        assert jefi.jefi_get_info(h)["device_status"] == 0
        jefi.jefi_destroy(h)


def test_plan_runs_interpolated_handles(gpu, plan_problems):
    """Second-order (JEFI_FLAG_INTERP) and floor-rule handles in one plan:
    replays equal jefi_eval_batch bit for bit, the interpolated entries match
    the oracle's second-order sum."""
    import torch

    probs, hists = plan_problems
    specs = [(1, "fp32c", jefi.JEFI_FLAG_INTERP), (2, "fp64", jefi.JEFI_FLAG_INTERP), (3, "fp64", 0),
             (4, "fp32c", jefi.JEFI_FLAG_INTERP | jefi.JEFI_FLAG_DIRECT_GATHER)]
    hs = []
    for k, prec, flags in specs:
        h = create(probs[k], prec, flags=flags)
        push_all(h, hists[k], upto=probs[k].n_push)
        hs.append(h)
    ts = []
    for h in hs:
        lo, hi = jefi.jefi_valid_window(h)
        ts.append(0.5 * (lo + hi) if np.isfinite(lo) else hi - 0.5 * probs[1].dt)
    outs = [_alloc(h) for h in hs]
    plan = jefi.jefi_batch_plan_create(hs, [o[0] for o in outs], [o[1] for o in outs])
    jefi.jefi_batch_plan_launch(plan, ts)
    torch.cuda.synchronize()
    _assert_equal(outs, _batch_reference(hs, ts))
    for (k, prec, flags), (E, B), t in zip(specs, outs, ts):
        p = probs[k]
        rho, J, _, _ = hists[k]
        n = p.n_push
        fn = oracle.fields_interp if flags & jefi.JEFI_FLAG_INTERP else oracle.fields
        Er, Br = fn(p.src.n, p.src.lo, p.src.d, p.obs(), rho[:n], J[:n], dt=p.dt, t0=p.t0, t=t)
        tol = 1e-12 if prec == "fp64" else 1e-5
        assert rel_l2(E.cpu().numpy(), Er) <= tol and rel_l2(B.cpu().numpy(), Br) <= tol, k
    jefi.jefi_batch_plan_destroy(plan)
    for h in hs:
        assert jefi.jefi_get_info(h)["device_status"] == 0
        jefi.jefi_destroy(h)


def test_tune_cache_round_trip(gpu, plan_problems, tmp_path, monkeypatch):
    """With JEFI_TUNE_CACHE set, a tuning stores its choice under the plan's
    geometry key; the same batch on fresh handles then takes the stored
    choice without timing candidates (from_cache), gives the same kernels and
    splits, and its results still match the oracle."""
    import torch

    path = tmp_path / "tune.txt"
    monkeypatch.setenv("JEFI_TUNE_CACHE", str(path))
    probs, hists = plan_problems
    ts = [p.times[0] for p in probs] + [probs[0].times[0]]
    chosen = []
    for round_ in range(2):
        hs, view = _handles(probs, hists)
        entries = hs + [view]
        outs = [_alloc(h) for h in entries]
        plan = jefi.jefi_batch_plan_create(entries, [o[0] for o in outs], [o[1] for o in outs])
        rep = jefi.jefi_batch_plan_tune(plan, ts)
        assert rep["from_cache"] == round_
        if round_ == 1:
            assert rep["candidates"] == 1
        chosen.append([(jefi.jefi_get_info(h)["staged_band"], jefi.jefi_get_info(h)["n_split"]) for h in entries])
        jefi.jefi_batch_plan_launch(plan, ts)
        torch.cuda.synchronize()
        _assert_equal(outs, _batch_reference(entries, ts))
        for k in range(len(hs)):
            _check_oracle(probs, hists, k, outs[k][0], outs[k][1], ts[k], probs[k].n_push)
        jefi.jefi_batch_plan_destroy(plan)
        for h in [view] + hs:
            jefi.jefi_destroy(h)
    assert chosen[0] == chosen[1]
    assert len(path.read_text().strip().splitlines()) == 1
