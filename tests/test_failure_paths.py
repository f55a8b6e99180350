"""Failure detection without faulting a GPU.

* Host side: an allocator callback that fails after N allocations makes
  jefi_create return JEFI_ENOMEM and release every earlier allocation (runs
  on CPU: no CUDA call happens before the allocations).
* Device side: a kernel waits on a barrier that nothing completes, through
  the bounded wait of the staged kernel; the wait expires, the status says
  JEFI_ETIMEOUT and the context stays usable.
"""
import ctypes

import numpy as np
import pytest

import paper_2104_05426_gb300 as jefi


class FailingAllocator:
    """Hands out host memory as fake device pointers until `budget` calls."""

    def __init__(self, budget):
        self.budget = budget
        self.live = {}
        self.calls = 0
        self.alloc = jefi.ALLOC_FN(self._alloc)
        self.free = jefi.FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        self.calls += 1
        if self.calls > self.budget:
            return None
        buf = ctypes.create_string_buffer(max(int(nbytes), 1))
        addr = ctypes.addressof(buf)
        self.live[addr] = buf
        return addr

    def _free(self, ptr, ctx):
        self.live.pop(ptr, None)


@pytest.mark.parametrize("budget", [0, 1, 3, 6])
def test_allocation_failure_releases_everything(budget):
    fa = FailingAllocator(budget)
    p = jefi.default_params(dt=0.1, history_slots=8)
    p.alloc = fa.alloc
    p.free = fa.free
    out = ctypes.c_void_p()
    g = jefi.grid((6, 5, 4), (0, 0, 0), (0.2,) * 3)
    pts = np.ascontiguousarray(np.random.default_rng(0).uniform(2, 3, (40, 3)))
    rc = jefi.load().jefi_create(ctypes.byref(g), None, pts.ctypes.data, 40, ctypes.byref(p), None,
                                 ctypes.byref(out))
    assert rc == jefi.JEFI_ENOMEM
    assert not out.value
    assert fa.calls > budget               # the failing call was reached
    assert fa.live == {}                   # every successful allocation was freed


@pytest.mark.gpu
def test_bounded_device_wait_reports_timeout(gpu):
    import torch

    assert jefi.jefi_debug_wait_timeout(0.05) == jefi.JEFI_ETIMEOUT
    # the context is still usable afterwards
    x = torch.arange(10, device="cuda", dtype=torch.float64)
    assert float(x.sum().item()) == 45.0
