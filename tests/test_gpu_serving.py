"""Serving loop: continuous batching of field-evaluation requests against
resident source problems.  Each result is bit-identical to evaluating the same
view at the same time alone; admission respects the memory budget; pushes
interleave safely with in-flight batches."""
import numpy as np
import pytest

import paper_2104_05426_gb300 as jefi
from paper_2104_05426_gb300.serving import ServingEngine, make_problems, poisson_requests

pytestmark = pytest.mark.gpu


def test_served_results_equal_single_evaluations(gpu):
    import torch

    probs = make_problems(3, seed=1, sides=(8, 14), H_range=(40, 56))
    eng = ServingEngine(probs, obs_half_width=2.0, n_streams=3, max_batch=8, tick_s=None,
                        keep_outputs=True)
    reqs = poisson_requests(48, rate=5000.0, n_problems=3, seed=3, side_choices=[4, 6, 8, 9])
    stats = eng.run(reqs)
    assert stats.completed == len(reqs) and stats.rejected == 0
    assert stats.max_batch > 1                       # requests were batched together
    for r in reqs:
        E = torch.empty_like(r.E)
        B = torch.empty_like(r.B)
        jefi.jefi_eval_fields(r.view[0], r.t, E, B)
        torch.cuda.synchronize()
        assert torch.equal(E, r.E) and torch.equal(B, r.B), r.rid
        assert jefi.jefi_get_info(r.view[0])["device_status"] == 0
    eng.close()


def test_serving_with_pushes_and_memory_budget(gpu):
    probs = make_problems(3, seed=2, sides=(8, 12), H_range=(40, 48))
    resident = sum(jefi.jefi_get_info(p.handle)["device_bytes"] for p in probs)
    budget = resident + 24 * (1 << 20)               # room for a few views at a time
    eng = ServingEngine(probs, obs_half_width=2.0, n_streams=2, max_batch=6, tick_s=0.003,
                        memory_budget=budget)
    reqs = poisson_requests(60, rate=800.0, n_problems=3, seed=4, side_choices=[4, 6, 8])
    stats = eng.run(reqs)
    assert stats.completed + stats.rejected == len(reqs)
    assert stats.evicted == 0 and stats.failed == 0   # times are placed in the window at launch
    assert stats.completed >= len(reqs) // 2
    assert stats.peak_bytes <= budget
    assert np.isfinite(stats.p50_ms) and stats.p99_ms >= stats.p50_ms
    eng.close()


def test_cached_view_is_not_evicted_under_its_own_request(gpu):
    """A request whose cached view is idle, admitted when the budget needs an
    eviction: the eviction must not take that view (the request would be
    launched on a destroyed handle).  Three requests on one stream, one at a
    time, under a budget that holds both views but only one output."""
    from paper_2104_05426_gb300.serving import Request

    probs = make_problems(1, seed=5, sides=(12, 12), H_range=(40, 40))
    p = probs[0]
    sizes = {}
    for s in (8, 12):
        v = jefi.jefi_create_view(p.handle, obs_grid=jefi.grid((s,) * 3, (-2.0,) * 3, (4.0 / s,) * 3))
        sizes[s] = jefi.jefi_get_info(v)["device_bytes"]
        jefi.jefi_destroy(v)
    out = {s: s ** 3 * 6 * 8 for s in (8, 12)}
    resident = jefi.jefi_get_info(p.handle)["device_bytes"]
    budget = resident + sizes[8] + sizes[12] + out[12] + out[8] // 2
    eng = ServingEngine(probs, obs_half_width=2.0, n_streams=1, max_batch=1, tick_s=None, memory_budget=budget)
    eng.view_bytes.update({(0, 8): sizes[8], (0, 12): sizes[12]})
    reqs = [Request(0, 0, 8, 0.5, 0.0), Request(1, 0, 12, 0.5, 0.0), Request(2, 0, 8, 0.5, 0.0)]
    stats = eng.run(reqs)
    assert stats.completed == 3 and stats.rejected == 0 and stats.failed == 0
    assert stats.peak_bytes <= budget
    assert eng.views_created == 2                    # the third request reused the first view
    eng.close()


def test_served_results_match_the_oracle(gpu):
    """A seeded sample of requests served under pushes, against the FP64 CPU
    oracle on the same history (slice n = the source model at n dt): the
    compensated FP32 contract, rel-L2 <= 1e-5 per field."""
    import math

    import oracle
    from paper_2104_05426_gb300.serving import served_sample
    from workloads import Grid

    probs = make_problems(2, seed=5, sides=(8, 12), H_range=(40, 48))
    eng = ServingEngine(probs, obs_half_width=2.0, n_streams=2, max_batch=6, tick_s=0.004,
                        keep_ids=range(0, 40, 5))
    reqs = poisson_requests(40, rate=600.0, n_problems=2, seed=6, side_choices=[5, 8, 10])
    stats = eng.run(reqs)
    assert stats.completed == len(reqs)
    samples = [served_sample(eng, r) for r in reqs if r.rid in eng.keep_ids]
    assert len(samples) == 8
    for sm in samples:
        src = Grid.cube(sm["src_side"], -sm["src_half_width"], sm["src_half_width"])
        obs = Grid.cube(sm["obs_side"], -sm["obs_half_width"], sm["obs_half_width"]).points()
        dt, t = sm["dt"], sm["t"]
        model = sm["model"]
        n_hi = sm["n_pushed"] - 1
        rmax = math.sqrt(3.0) * (sm["src_half_width"] + sm["obs_half_width"])
        n_lo = max(0, int(math.floor((t - rmax) / dt)) - 2)
        hist = [model.sample(src, n * dt) for n in range(n_lo, n_hi + 1)]
        rho = np.stack([h[0] for h in hist])
        J = np.stack([h[1] for h in hist])
        Er, Br = oracle.fields(src.n, src.lo, src.d, obs, rho, J, dt=dt, t0=n_lo * dt, t=t)
        for got, ref in ((sm["E"], Er), (sm["B"], Br)):
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5, sm["rid"]
    eng.close()
