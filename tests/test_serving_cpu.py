"""Host logic of the serving loop that needs no GPU: the seeded Poisson
request stream the serving measurements are quoted on (arrival rate,
determinism, the ranges of problems, observation sides and window
positions)."""
import numpy as np

from paper_2104_05426_gb300.serving import poisson_requests


def test_poisson_stream_rate_and_ranges():
    reqs = poisson_requests(20000, rate=80.0, n_problems=64, obs_sides=(8, 48), seed=3)
    arr = np.array([r.arrival for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert np.all(gaps > 0)                                   # arrivals strictly increase
    assert abs(gaps.mean() * 80.0 - 1.0) < 0.03               # mean gap 1/rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05         # exponential: cv = 1
    assert {r.problem for r in reqs} == set(range(64))
    sides = [r.obs_side for r in reqs]
    assert min(sides) == 8 and max(sides) == 48
    fr = np.array([r.frac for r in reqs])
    assert fr.min() >= 0.05 and fr.max() <= 0.95
    assert [r.rid for r in reqs] == list(range(20000))


def test_poisson_stream_is_seeded():
    a = poisson_requests(500, rate=10.0, n_problems=8, seed=11, side_choices=[8, 16, 24])
    b = poisson_requests(500, rate=10.0, n_problems=8, seed=11, side_choices=[8, 16, 24])
    c = poisson_requests(500, rate=10.0, n_problems=8, seed=12, side_choices=[8, 16, 24])
    key = lambda rs: [(r.problem, r.obs_side, r.frac, r.arrival) for r in rs]
    assert key(a) == key(b) and key(a) != key(c)
    assert {r.obs_side for r in a} == {8, 16, 24}
