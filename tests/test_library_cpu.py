"""CPU checks of libjefi: it builds, loads, exports every declared symbol, and
its host-side exact slot rule agrees with the oracle's (no GPU needed)."""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
import paper_2104_05426_gb300 as jefi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(jefi_\w+)\s*\(", text, flags=re.M):
                names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = jefi._build.build()
    L = jefi.load()
    declared = declared_functions()
    assert declared, "no declarations found"
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (jefi_\w+)", out))
    missing = declared - exported
    assert not missing, missing
    for name in declared:
        getattr(L, name)
    assert set(jefi.EXPORTS) == declared


def test_strerror_and_defaults():
    assert jefi.strerror(0) == "ok"
    assert "pushed" in jefi.strerror(jefi.JEFI_ENOTYET)
    p = jefi.default_params()
    assert p.c == 1.0 and p.history_slots == 64 and p.precision == jefi.JEFI_FP32_COMP
    assert list(p.screen) == [-1.0, -1.0, -1.0]


def test_host_slot_rule_matches_oracle_random_pairs():
    rng = np.random.Generator(np.random.PCG64(3))
    for c, dt, t, t0 in ((1.0, 0.0625, 7.3, 0.0), (2.7, 0.1, 31.1, -4.2), (0.3, 0.013, 3.0, 1.0)):
        xo = rng.uniform(-6, 6, (20000, 3))
        xs = rng.uniform(-6, 6, (20000, 3))
        a = jefi.jefi_host_pair_slots(xo, xs, t, t0, c, dt)
        b = oracle.pair_slots(xo, xs, t=t, t0=t0, c=c, dt=dt)
        assert np.array_equal(a, b)


def test_host_slot_rule_matches_oracle_on_ties():
    """Dyadic pairs whose u is an exact integer, and their neighbours."""
    offs = np.array([[1, 2, 2], [2, 3, 6], [1, 4, 8], [0, 3, 4], [6, 6, 7]], float)
    rs = np.array([3, 7, 9, 5, 11], float)
    xs = np.tile([[0.25, -0.5, 1.0]], (len(offs), 1))
    for s in (0.125, 0.5):
        xo = xs + offs * s
        for dt in (0.0625, 0.125):
            for k in (0, 5, 40):
                for eps in (0.0, dt / 8, -dt / 8):
                    t = k * dt + rs * s
                    for i in range(len(offs)):
                        a = jefi.jefi_host_pair_slots(xo[i:i + 1], xs[i:i + 1], t[i] + eps, 0.0, 1.0, dt)
                        b = oracle.pair_slots(xo[i:i + 1], xs[i:i + 1], t=t[i] + eps, t0=0.0, c=1.0, dt=dt)
                        assert a[0] == b[0]


def test_handle_creation_without_gpu_fails_cleanly():
    """Without a CUDA device the library reports an error code instead of
    falling back to anything."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    g = jefi.grid((4, 4, 4), (0, 0, 0), (0.25,) * 3)
    with pytest.raises(jefi.JefiError) as e:
        jefi.jefi_create(g, obs_points=np.zeros((5, 3)) + 3.0,
                         params=jefi.default_params(dt=0.1, history_slots=8), stream=0)
    assert e.value.code in (jefi.JEFI_ENOMEM, jefi.JEFI_ECUDA)


def test_batch_plan_entry_points_reject_bad_arguments():
    """Argument checks of the batch-plan calls happen before any CUDA call."""
    import ctypes

    L = jefi.load()
    out = ctypes.c_void_p()
    assert L.jefi_batch_plan_create(None, None, None, -1, ctypes.byref(out)) == jefi.JEFI_EINVAL
    assert L.jefi_batch_plan_create(None, None, None, 1, ctypes.byref(out)) == jefi.JEFI_EINVAL
    assert L.jefi_batch_plan_create(None, None, None, 0, None) == jefi.JEFI_EINVAL
    assert L.jefi_batch_plan_launch(None, None, None) == jefi.JEFI_EINVAL
    assert L.jefi_batch_plan_tune(None, None, None, None) == jefi.JEFI_EINVAL
    assert L.jefi_batch_plan_destroy(None) == jefi.JEFI_EINVAL
    with pytest.raises(ValueError):                   # one output pair per handle
        jefi.jefi_batch_plan_create([object()], [], [])
    with pytest.raises(ValueError):                   # outputs must be device tensors
        jefi.jefi_batch_plan_create([object()], [np.zeros((1, 3))], [np.zeros((1, 3))])


def test_no_cpu_fallback_without_a_device():
    """Without a CUDA device every compute entry fails with an error code:
    there is no CPU path behind the C ABI."""
    import ctypes

    import torch

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    L = jefi.load()
    g = jefi.grid((4, 4, 4), (0.0,) * 3, (0.25,) * 3)
    obs = jefi.grid((4, 4, 4), (2.0,) * 3, (0.25,) * 3)
    with pytest.raises(jefi.JefiError) as e:
        jefi.jefi_create(g, obs_grid=obs, params=jefi.default_params(dt=0.1, history_slots=8))
    assert e.value.code in (jefi.JEFI_ENOMEM, jefi.JEFI_ECUDA)
    assert jefi.jefi_debug_wait_timeout(0.01) == jefi.JEFI_ECUDA
    out = ctypes.c_void_p()
    assert L.jefi_batch_plan_create(None, None, None, 0, ctypes.byref(out)) == jefi.JEFI_ECUDA
    assert not out.value


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "jefi.h"

/* every entry point, by address: the header must declare them all for C */
typedef void (*entry_fn)(void);
static const entry_fn entries[] = {
    (entry_fn)jefi_default_params, (entry_fn)jefi_create, (entry_fn)jefi_create_view, (entry_fn)jefi_push_sources,
    (entry_fn)jefi_eval_fields, (entry_fn)jefi_eval_fields_multi, (entry_fn)jefi_eval_batch,
    (entry_fn)jefi_valid_window, (entry_fn)jefi_get_info, (entry_fn)jefi_reset_stats, (entry_fn)jefi_debug_slots,
    (entry_fn)jefi_debug_wait_timeout, (entry_fn)jefi_host_pair_slots, (entry_fn)jefi_eval_fields_noalloc,
    (entry_fn)jefi_checkpoint_bytes, (entry_fn)jefi_checkpoint, (entry_fn)jefi_restore, (entry_fn)jefi_select_kernel,
    (entry_fn)jefi_batch_plan_create, (entry_fn)jefi_batch_plan_launch, (entry_fn)jefi_batch_plan_tune,
    (entry_fn)jefi_batch_plan_destroy, (entry_fn)jefi_destroy, (entry_fn)jefi_strerror};

int main(void) {
    jefi_params p;
    jefi_default_params(&p);
    double xo[3] = {3.0, 4.0, 0.0}, xs[3] = {0.0, 0.0, 0.0};
    int64_t slot = -1;
    jefi_host_pair_slots(1, xo, xs, 10.0, 0.0, 1.0, 0.5, &slot);   /* floor((10 - 5)/0.5) = 10 */
    printf("%d %d %s %lld %d\n", (int)(sizeof(entries) / sizeof(entries[0])), p.history_slots,
           jefi_strerror(JEFI_OK), (long long)slot, jefi_destroy(NULL));
    return 0;
}
"""


def test_header_is_c99_and_the_library_links_from_c(tmp_path):
    """include/jefi.h compiles as C99 with warnings as errors, a C program
    links libjefi.so and calls the entry points that need no device."""
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    lib_dir = os.path.dirname(jefi._build.build())
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", lib_dir, "-l:libjefi.so", "-Wl,-rpath," + lib_dir],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert out == ["24", "64", "ok", "10", str(jefi.JEFI_EINVAL)]


def test_noalloc_wrapper_checks_shapes_before_any_launch():
    """The allocation-free entry cannot see the sizes of device buffers, so the
    binding checks every shape against the grid before anything is launched
    (host arrays here: the shape error comes before the device check)."""
    g = jefi.grid((3, 4, 5), (0.0,) * 3, (0.1,) * 3)        # N_src = 60
    prm = jefi.default_params(dt=0.1)
    obs, rho, J = np.zeros((7, 3)), np.zeros((4, 60)), np.zeros((4, 60, 3))
    E, B = np.zeros((7, 3)), np.zeros((7, 3))
    bad = [
        dict(obs=np.zeros((7, 2))),
        dict(obs=np.zeros(21)),
        dict(rho=np.zeros((4, 59))),
        dict(rho=np.zeros(240)),
        dict(J=np.zeros((4, 60, 2))),
        dict(J=np.zeros((3, 60, 3))),
        dict(E=np.zeros((6, 3))),
        dict(B=np.zeros((7, 3, 1))),
    ]
    for change in bad:
        args = dict(obs=obs, rho=rho, J=J, E=E, B=B)
        args.update(change)
        with pytest.raises(ValueError, match="shape"):
            jefi.jefi_eval_fields_noalloc(g, args["obs"], args["rho"], args["J"], prm, 1.0, args["E"], args["B"])
    with pytest.raises(ValueError, match="device"):     # right shapes, host buffers
        jefi.jefi_eval_fields_noalloc(g, obs, rho, J, prm, 1.0, E, B)


def _wave_cost(units, n_split, bps, resident):
    """Waves x (bricks per item + half a brick of preamble) of the least
    costly merge, by brute force over every merge (the rule the library
    searches in O(sqrt(n_split)) steps)."""
    best = None
    for m in range(1, n_split + 1):
        items = units * -(-n_split // m)
        c = -(-items // resident) * (m * bps + 0.5)
        if best is None or c < best[0]:
            best = (c, m)
    return best


def test_split_plan_fills_whole_waves():
    """The dipole workload (16 tiles, 512 bricks, 4 times per launch) and a
    64^3-source view of 32^3 points: creation picks the split counts whose
    launches run whole waves of equal items on 304 CTA slots."""
    assert jefi.jefi_host_split_plan(16, 512, 170, 8, 304) == (19, 27, 1)
    n, bps, m = jefi.jefi_host_split_plan(128, 4096, 10, 2, 304)
    assert (n, bps, m) == (7, 586, 1)
    assert 128 * n / (-(-128 * n // 304) * 304) > 0.98     # items fill 98 % of their waves


def test_split_plan_is_consistent_and_optimal():
    rng = np.random.Generator(np.random.PCG64(21))
    for _ in range(300):
        tiles = int(rng.integers(1, 2000))
        bricks = int(rng.integers(1, 5000))
        cap = int(rng.integers(1, 300))
        chunk = int(rng.choice([1, 2, 8]))
        resident = int(rng.choice([152, 304, 456]))
        n, bps, m = jefi.jefi_host_split_plan(tiles, bricks, cap, chunk, resident)
        assert 1 <= n <= min(cap, bricks) and bps * (n - 1) < bricks <= bps * n
        assert m == _wave_cost(tiles, n, bps, resident)[1]
        # no other count within the cap predicts less time, averaged over
        # launches of 1, 2, 4, ... chunk times
        ts = [1]
        while ts[-1] < chunk:
            ts.append(min(2 * ts[-1], chunk))

        def score(k):
            b = -(-bricks // k)
            kk = -(-bricks // b)
            return sum(_wave_cost(tiles * t, kk, b, resident)[0] / (tiles * t * bricks / resident)
                       for t in ts) / len(ts)

        if cap <= 60:
            chosen = score(n)
            assert all(chosen <= score(k) + 1e-9 for k in range(1, min(cap, bricks) + 1))


def test_split_plan_rejects_bad_arguments():
    for args in ((0, 10, 5, 1, 304), (4, 0, 5, 1, 304), (4, 10, 0, 1, 304), (4, 10, 5, 0, 304),
                 (4, 10, 5, 1, 0)):
        with pytest.raises(jefi.JefiError):
            jefi.jefi_host_split_plan(*args)
