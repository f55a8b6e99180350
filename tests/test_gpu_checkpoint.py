"""Checkpoint and resume of a handle's resident history (jefi_checkpoint /
jefi_restore) through the C ABI.

A restored handle must behave exactly like one that received every slice by
push: bit-identical fields now, and after further pushes (the difference
state is part of the image), whatever its observation points.
"""
import numpy as np
import pytest

import paper_2104_05426_gb300 as jefi
from jefi_cases import create, history
from workloads import Blob, Grid, MovingGaussians, Problem

pytestmark = pytest.mark.gpu


def problem(obs_grid, n_push=100, H=40):
    src = Grid((10, 9, 7), (-0.5, -0.45, -0.35), (0.1, 0.1, 0.1))
    blob = Blob(1.0, (0.15, 0.2, 0.15), (-0.2, 0.0, 0.0), (0.25, 0.05, 0.0))
    return Problem("ckp", src, obs_grid, None, 0.0625, H, n_push, [],
                   MovingGaussians([blob], noise=0.03, seed=8))


OBS_A = Grid.box((8, 8, 8), (1.0, -0.5, -0.5), (2.0, 0.5, 0.5))
OBS_B = Grid.box((12, 5, 9), (-0.6, 1.1, -0.7), (0.7, 2.5, 0.6))   # other tiles, other band


def fields(h, times):
    import torch

    E, B = jefi.eval_fields(h, np.asarray(times, dtype=np.float64))
    torch.cuda.synchronize()
    return E, B


def push_range(h, hist, lo, hi):
    import torch

    rho, J, _, _ = hist
    for n in range(lo, hi):
        jefi.jefi_push_sources(h, torch.from_numpy(rho[n]).cuda(), torch.from_numpy(J[n]).cuda())


@pytest.mark.parametrize("prec,flags", [("fp64", 0), ("fp32c", 0), ("fp32c", jefi.JEFI_FLAG_INTERP),
                                        ("fp64", jefi.JEFI_FLAG_INTERP)])
def test_restored_handle_equals_pushed_handle(gpu, prec, flags):
    import torch

    pa, pb = problem(OBS_A, n_push=107), problem(OBS_B, n_push=107)
    hist = history(pa)
    h1 = create(pa, prec, flags=flags)
    push_range(h1, hist, 0, 100)                  # the 40-slice ring has wrapped
    image = jefi.jefi_checkpoint(h1)
    h2 = create(pb, prec, flags=flags)            # other observation points
    push_range(h2, hist, 0, 3)                    # some unrelated state, overwritten
    jefi.jefi_restore(h2, image)
    h3 = create(pb, prec, flags=flags)
    push_range(h3, hist, 0, 100)
    assert jefi.jefi_valid_window(h2) == jefi.jefi_valid_window(h3)
    lo, hi = jefi.jefi_valid_window(h3)
    times = [lo, 0.5 * (lo + hi), hi]
    for a, b in zip(fields(h2, times), fields(h3, times)):
        assert torch.equal(a, b)
    # the difference state travelled too: the next slices continue identically
    push_range(h2, hist, 100, 107)
    push_range(h3, hist, 100, 107)
    lo, hi = jefi.jefi_valid_window(h3)
    times = [lo, 0.5 * (lo + hi), hi]
    for a, b in zip(fields(h2, times), fields(h3, times)):
        assert torch.equal(a, b)
    for h in (h1, h2, h3):
        assert jefi.jefi_get_info(h)["device_status"] == 0
        jefi.jefi_destroy(h)


def test_restore_refuses_foreign_or_damaged_images(gpu):
    import torch

    p = problem(OBS_A)
    hist = history(p)
    h = create(p, "fp32c")
    push_range(h, hist, 0, 60)
    image = jefi.jefi_checkpoint(h)
    lo, hi = jefi.jefi_valid_window(h)
    before = fields(h, [hi])

    def refused(target, img):
        with pytest.raises(jefi.JefiError) as e:
            jefi.jefi_restore(target, img)
        assert e.value.code == jefi.JEFI_EINVAL

    refused(h, image[:-1])                                   # truncated
    refused(h, b"X" + image[1:])                             # not an image
    other = create(problem(OBS_A, H=41), "fp32c")            # another history length
    refused(other, image)
    other64 = create(p, "fp64")                              # another precision
    refused(other64, image)
    view = jefi.jefi_create_view(h, obs_grid=jefi.grid_from(OBS_B))
    refused(view, image)                                     # views hold no history
    with pytest.raises(jefi.JefiError):
        jefi.jefi_checkpoint(view)
    # h is unchanged by the refusals
    assert jefi.jefi_valid_window(h) == (lo, hi)
    for a, b in zip(before, fields(h, [hi])):
        assert torch.equal(a, b)
    jefi.jefi_destroy(view)
    for x in (other, other64, h):
        jefi.jefi_destroy(x)


def test_views_of_a_restored_base_see_the_history(gpu):
    import torch

    p = problem(OBS_A)
    hist = history(p)
    h1 = create(p, "fp32c", flags=jefi.JEFI_FLAG_SHARED_RING)
    push_range(h1, hist, 0, 90)
    image = jefi.jefi_checkpoint(h1)
    h2 = create(p, "fp32c", flags=jefi.JEFI_FLAG_SHARED_RING)
    jefi.jefi_restore(h2, image)
    v1 = jefi.jefi_create_view(h1, obs_grid=jefi.grid_from(OBS_B))
    v2 = jefi.jefi_create_view(h2, obs_grid=jefi.grid_from(OBS_B))
    lo, hi = jefi.jefi_valid_window(v1)
    assert jefi.jefi_valid_window(v2) == (lo, hi)
    for a, b in zip(fields(v1, [lo, hi]), fields(v2, [lo, hi])):
        assert torch.equal(a, b)
    for x in (v1, v2, h1, h2):
        jefi.jefi_destroy(x)
