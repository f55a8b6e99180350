"""Python binding of libjefi: GB300 Jefimenko field evaluation (JefiGPU, Sec. 2.2).

Thin ctypes layer over the C ABI in ``include/jefi.h``: every function has
the C name and only marshals arguments (NumPy arrays for host memory, torch
CUDA tensors for device memory, torch streams).  All computation happens in
the CUDA kernels of ``libjefi.so``; there is no CPU path.  Importing this
package never falls back: if the library cannot be built or loaded, ``load``
raises.

Typical use::

    import paper_2104_05426_gb300 as jefi
    p = jefi.default_params(dt=0.0625, history_slots=80)
    h = jefi.jefi_create(jefi.grid((16,16,16), (-1,-1,-1), (0.125,)*3), obs_points=pts, params=p)
    jefi.jefi_push_sources(h, rho, J)           # numpy (host) or torch CUDA tensors
    E, B = jefi.eval_fields(h, t)               # torch CUDA tensors [N_obs, 3] FP64
    jefi.jefi_destroy(h)
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import build as _build

JEFI_OK = 0
JEFI_EINVAL = 1
JEFI_ENOMEM = 2
JEFI_ENOTYET = 3
JEFI_EEVICTED = 4
JEFI_ECUDA = 5
JEFI_ETIMEOUT = 6
JEFI_EINTERNAL = 7
JEFI_EUNSUPPORTED = 8

JEFI_FP64 = 0
JEFI_FP32 = 1
JEFI_FP32_COMP = 2
JEFI_DERIV_BACKWARD = 0
JEFI_DERIV_SUPPLIED = 1
JEFI_FLAG_STATS = 1
JEFI_FLAG_DIRECT_GATHER = 2
JEFI_FLAG_SHARED_RING = 4
JEFI_FLAG_INTERP = 8
JEFI_KERNEL_MEASURE = 0
JEFI_KERNEL_DIRECT = 1
JEFI_KERNEL_STAGED = 2

# Observation-grid tile shapes (points per tile along x, y, z); 0 = chosen at
# creation; 9 = packed (4x4x2-point blocks in Morton order, eight per tile)
TILE_SHAPES = {0: None, 1: (8, 8, 4), 2: (16, 4, 4), 3: (4, 8, 8), 4: (8, 4, 8), 5: (4, 16, 4),
               6: (16, 8, 2), 7: (8, 16, 2), 8: (4, 4, 16), 9: "packed"}
JEFI_TILE_PACKED = 9

PRECISIONS = {"fp64": JEFI_FP64, "fp32": JEFI_FP32, "fp32c": JEFI_FP32_COMP}

# Every symbol include/jefi.h declares (checked by the CPU test suite).
EXPORTS = ("jefi_default_params", "jefi_create", "jefi_push_sources", "jefi_eval_fields",
           "jefi_eval_fields_multi", "jefi_valid_window", "jefi_get_info", "jefi_reset_stats",
           "jefi_debug_slots", "jefi_host_pair_slots", "jefi_destroy", "jefi_strerror",
           "jefi_eval_fields_noalloc", "jefi_eval_batch", "jefi_create_view",
           "jefi_debug_wait_timeout", "jefi_checkpoint_bytes", "jefi_checkpoint", "jefi_restore",
           "jefi_select_kernel", "jefi_batch_plan_create", "jefi_batch_plan_launch",
           "jefi_batch_plan_tune", "jefi_batch_plan_destroy", "jefi_push_sources_region",
           "jefi_so_partition", "jefi_sum_fields", "jefi_host_split_plan")

JEFI_NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


class JefiError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} (code {code})")


class jefi_grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32 * 3), ("lo", ctypes.c_double * 3), ("d", ctypes.c_double * 3)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class jefi_params(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("k_e", ctypes.c_double), ("k_b", ctypes.c_double),
                ("dt", ctypes.c_double), ("t0", ctypes.c_double),
                ("history_slots", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("deriv", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("screen", ctypes.c_double * 3),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p),
                ("src_origin", ctypes.c_int32 * 3), ("tile_shape", ctypes.c_int32)]


class jefi_info(ctypes.Structure):
    _fields_ = [("n_src", ctypes.c_int64), ("n_obs", ctypes.c_int64), ("n_latest", ctypes.c_int64),
                ("pairs_per_eval", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("slot_fallbacks", ctypes.c_int64),
                ("sum_launches", ctypes.c_int64), ("sum_ms_total", ctypes.c_double),
                ("n_split", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("device_status", ctypes.c_int32), ("staged_band", ctypes.c_int32),
                ("tile_shape", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class jefi_tune_report(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int32), ("split_divisor", ctypes.c_int32),
                ("measured_kernels", ctypes.c_int32), ("staged_problems", ctypes.c_int32),
                ("concurrent_groups", ctypes.c_int32),
                ("ms_initial", ctypes.c_double), ("ms_tuned", ctypes.c_double),
                ("from_cache", ctypes.c_int32), ("widened_bands", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libjefi.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_needed and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libjefi.so is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(_build.LIB)
        P, I, I32, I64, D = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int32, ctypes.c_int64,
                             ctypes.c_double)
        L.jefi_default_params.argtypes = [ctypes.POINTER(jefi_params)]
        L.jefi_default_params.restype = None
        L.jefi_create.argtypes = [ctypes.POINTER(jefi_grid), ctypes.POINTER(jefi_grid), P, I64,
                                  ctypes.POINTER(jefi_params), P, ctypes.POINTER(P)]
        L.jefi_push_sources.argtypes = [P, P, P, P, P, I, P]
        L.jefi_eval_fields.argtypes = [P, D, P, P, I, P]
        L.jefi_eval_fields_multi.argtypes = [P, I32, P, P, P, I, P]
        L.jefi_valid_window.argtypes = [P, ctypes.POINTER(D), ctypes.POINTER(D)]
        L.jefi_get_info.argtypes = [P, ctypes.POINTER(jefi_info)]
        L.jefi_reset_stats.argtypes = [P]
        L.jefi_debug_slots.argtypes = [P, D, P, P]
        L.jefi_host_pair_slots.argtypes = [I64, P, P, D, D, D, D, P]
        L.jefi_host_pair_slots.restype = None
        PI32 = ctypes.POINTER(I32)
        L.jefi_host_split_plan.argtypes = [I64, I64, I64, I32, I64, PI32, PI32, PI32]
        L.jefi_destroy.argtypes = [P]
        L.jefi_eval_batch.argtypes = [P, P, P, P, I32, P]
        L.jefi_create_view.argtypes = [P, ctypes.POINTER(jefi_grid), P, I64, P, ctypes.POINTER(P)]
        L.jefi_create_view.restype = I
        L.jefi_debug_wait_timeout.argtypes = [D, P]
        L.jefi_debug_wait_timeout.restype = I
        L.jefi_eval_batch.restype = I
        L.jefi_eval_fields_noalloc.argtypes = [ctypes.POINTER(jefi_grid), P, I64, P, P, I64,
                                               ctypes.POINTER(jefi_params), D, P, P, P]
        L.jefi_eval_fields_noalloc.restype = I
        L.jefi_checkpoint_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
        L.jefi_checkpoint.argtypes = [P, P, ctypes.c_size_t, P]
        L.jefi_restore.argtypes = [P, P, ctypes.c_size_t, P]
        L.jefi_select_kernel.argtypes = [P, I32, D, ctypes.POINTER(I32), P]
        L.jefi_select_kernel.restype = I
        L.jefi_batch_plan_create.argtypes = [P, P, P, I32, ctypes.POINTER(P)]
        L.jefi_batch_plan_launch.argtypes = [P, P, P]
        L.jefi_batch_plan_tune.argtypes = [P, P, P, ctypes.POINTER(jefi_tune_report)]
        L.jefi_batch_plan_destroy.argtypes = [P]
        for name in ("jefi_batch_plan_create", "jefi_batch_plan_launch", "jefi_batch_plan_tune",
                     "jefi_batch_plan_destroy"):
            getattr(L, name).restype = I
        L.jefi_push_sources_region.argtypes = [P, P, P, P, P, ctypes.POINTER(I32), ctypes.POINTER(I32), I, P]
        L.jefi_push_sources_region.restype = I
        L.jefi_so_partition.argtypes = [ctypes.POINTER(jefi_grid), ctypes.POINTER(I32), ctypes.POINTER(jefi_grid),
                                        ctypes.POINTER(I32)]
        L.jefi_so_partition.restype = I
        L.jefi_sum_fields.argtypes = [I32, P, P, I64, P, P, P]
        L.jefi_sum_fields.restype = I
        L.jefi_strerror.argtypes = [I]
        L.jefi_strerror.restype = ctypes.c_char_p
        for name in ("jefi_create", "jefi_push_sources", "jefi_eval_fields",
                     "jefi_eval_fields_multi", "jefi_valid_window", "jefi_get_info",
                     "jefi_reset_stats", "jefi_debug_slots", "jefi_destroy"):
            getattr(L, name).restype = I
        _lib = L
        return L


def strerror(code: int) -> str:
    try:
        return load().jefi_strerror(int(code)).decode()
    except Exception:  # pragma: no cover - only when the library itself is missing
        return "unknown"


def _check(rc: int, what: str):
    if rc != JEFI_OK:
        raise JefiError(rc, what)


# ---------------------------------------------------------------------------- marshalling
def grid(n: Sequence[int], lo: Sequence[float], d: Sequence[float]) -> jefi_grid:
    g = jefi_grid()
    for a in range(3):
        g.n[a] = int(n[a])
        g.lo[a] = float(lo[a])
        g.d[a] = float(d[a])
    return g


def grid_from(obj) -> jefi_grid:
    """From any object with ``n``, ``lo`` and ``d`` attributes (e.g. workloads.Grid)."""
    return grid(obj.n, obj.lo, obj.d)


def default_params(**kw) -> jefi_params:
    p = jefi_params()
    load().jefi_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "screen":
            for a in range(3):
                p.screen[a] = float(v[a])
            continue
        if k == "src_origin":
            for a in range(3):
                p.src_origin[a] = int(v[a])
            continue
        setattr(p, k, v)
    return p


class _TorchAllocator:
    """Device allocations through torch's caching allocator (kept alive by the handle)."""

    def __init__(self):
        import torch

        self._torch = torch
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            return self._torch.cuda.caching_allocator_alloc(int(nbytes))
        except Exception:
            return None

    def _free(self, ptr, ctx):
        self._torch.cuda.caching_allocator_delete(ptr)


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _buf(x, dtype=np.float64):
    """(pointer, on_device, keepalive) for a numpy array or torch tensor."""
    if x is None:
        return None, None, None
    try:
        import torch

        if isinstance(x, torch.Tensor):
            if x.dtype != torch.float64 or not x.is_contiguous():
                raise ValueError("tensors must be contiguous float64")
            return x.data_ptr(), bool(x.is_cuda), x
    except ImportError:  # pragma: no cover
        pass
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, False, a


class Handle:
    """Owns a jefi_handle plus the Python objects its callbacks need."""

    def __init__(self, ptr, keep):
        self.ptr = ptr
        self._keep = keep
        self.n_obs = 0
        self.n_src = 0

    @property
    def value(self):
        return self.ptr.value


# ---------------------------------------------------------------------------- C names
def jefi_create(src: jefi_grid, obs_grid: Optional[jefi_grid] = None, obs_points=None,
                params: Optional[jefi_params] = None, stream=None, torch_allocator: bool = False):
    L = load()
    if params is None:
        params = default_params()
    keep = []
    if torch_allocator:
        ta = _TorchAllocator()
        params.alloc = ta.alloc
        params.free = ta.free
        keep.append(ta)
    pts_ptr, n_obs = None, 0
    if obs_grid is None:
        pts = np.ascontiguousarray(obs_points, dtype=np.float64).reshape(-1, 3)
        pts_ptr, n_obs = pts.ctypes.data, pts.shape[0]
        keep.append(pts)
    out = ctypes.c_void_p()
    rc = L.jefi_create(ctypes.byref(src), ctypes.byref(obs_grid) if obs_grid is not None else None,
                       pts_ptr, n_obs, ctypes.byref(params), _stream_ptr(stream), ctypes.byref(out))
    _check(rc, "jefi_create")
    keep.append(params)
    h = Handle(out, keep)
    info = jefi_get_info(h)
    h.n_obs = int(info["n_obs"])
    h.n_src = int(info["n_src"])
    return h


def jefi_push_sources(h: Handle, rho, J, drho_dt=None, dJ_dt=None, stream=None):
    r, on_dev, k1 = _buf(rho)
    j, on_dev_j, k2 = _buf(J)
    dr, _, k3 = _buf(drho_dt)
    dj, _, k4 = _buf(dJ_dt)
    if on_dev_j is not None and on_dev is not None and on_dev != on_dev_j:
        raise ValueError("rho and J must both be host or both device buffers")
    rc = load().jefi_push_sources(h.ptr, r, j, dr, dj, 1 if on_dev else 0, _stream_ptr(stream))
    _check(rc, "jefi_push_sources")


def jefi_push_sources_region(h: Handle, rho, J, full_n, offset, drho_dt=None, dJ_dt=None, stream=None):
    """Push one slice whose arrays cover the grid full_n (x fastest); the
    handle's cell (i, j, k) is their cell offset + (i, j, k)."""
    r, on_dev, k1 = _buf(rho)
    j, on_dev_j, k2 = _buf(J)
    dr, _, k3 = _buf(drho_dt)
    dj, _, k4 = _buf(dJ_dt)
    if on_dev_j is not None and on_dev is not None and on_dev != on_dev_j:
        raise ValueError("rho and J must both be host or both device buffers")
    n_full = int(full_n[0]) * int(full_n[1]) * int(full_n[2])
    for name, x, per in (("rho", rho, 1), ("J", J, 3), ("drho_dt", drho_dt, 1), ("dJ_dt", dJ_dt, 3)):
        if x is not None and int(np.prod(x.shape)) != per * n_full:
            raise ValueError(f"{name} must hold {per} x {n_full} values for the grid {tuple(full_n)}")
    fn = (ctypes.c_int32 * 3)(*[int(v) for v in full_n])
    off = (ctypes.c_int32 * 3)(*[int(v) for v in offset])
    rc = load().jefi_push_sources_region(h.ptr, r, j, dr, dj, fn, off, 1 if on_dev else 0, _stream_ptr(stream))
    _check(rc, "jefi_push_sources_region")


def jefi_so_partition(src: jefi_grid, parts):
    """The source grid cut into parts[0] x parts[1] x parts[2] brick-aligned
    boxes (x fastest): a list of (sub-grid, origin) -- create each box's
    handle with default_params(..., src_origin=origin)."""
    n = int(parts[0]) * int(parts[1]) * int(parts[2])
    if n < 1:
        raise ValueError("parts must be positive")
    sub = (jefi_grid * n)()
    org = (ctypes.c_int32 * (3 * n))()
    p = (ctypes.c_int32 * 3)(*[int(v) for v in parts])
    _check(load().jefi_so_partition(ctypes.byref(src), p, sub, org), "jefi_so_partition")
    return [(sub[k], (org[3 * k], org[3 * k + 1], org[3 * k + 2])) for k in range(n)]


def jefi_sum_fields(E_parts, B_parts, E, B, stream=None):
    """E = E_parts[0] + E_parts[1] + ... (FP64, in list order), the same for
    B; all CUDA float64 tensors of one shape [n_obs, 3]."""
    n = len(E_parts)
    if n != len(B_parts) or n < 1:
        raise ValueError("E_parts and B_parts must be non-empty lists of the same length")
    shape = tuple(E.shape)
    ptrs_e, ptrs_b = [], []
    for x in list(E_parts) + list(B_parts) + [E, B]:
        if tuple(x.shape) != shape:
            raise ValueError(f"every field array must have the shape {shape}")
    for x_list, ptrs in ((E_parts, ptrs_e), (B_parts, ptrs_b)):
        for x in x_list:
            p, on_dev, _ = _buf(x)
            if not on_dev:
                raise ValueError("jefi_sum_fields takes device (CUDA) tensors only")
            ptrs.append(p)
    e, on_e, _ = _buf(E)
    bb, on_b, _ = _buf(B)
    if not (on_e and on_b):
        raise ValueError("jefi_sum_fields takes device (CUDA) tensors only")
    pe = (ctypes.c_void_p * n)(*ptrs_e)
    pb = (ctypes.c_void_p * n)(*ptrs_b)
    n_obs = int(np.prod(shape)) // 3
    _check(load().jefi_sum_fields(n, pe, pb, n_obs, e, bb, _stream_ptr(stream)), "jefi_sum_fields")


def jefi_eval_fields(h: Handle, t: float, E, B, stream=None):
    e, on_dev, ke = _buf(E)
    b, _, kb = _buf(B)
    if not on_dev and (ke is not E or kb is not B):
        raise ValueError("host outputs must be contiguous float64 numpy arrays")
    rc = load().jefi_eval_fields(h.ptr, float(t), e, b, 1 if on_dev else 0, _stream_ptr(stream))
    _check(rc, "jefi_eval_fields")


def jefi_eval_fields_multi(h: Handle, times, E, B, stream=None):
    ts = np.ascontiguousarray(times, dtype=np.float64).reshape(-1)
    e, on_dev, ke = _buf(E)
    b, _, kb = _buf(B)
    if not on_dev and (ke is not E or kb is not B):
        raise ValueError("host outputs must be contiguous float64 numpy arrays")
    rc = load().jefi_eval_fields_multi(h.ptr, ts.shape[0], ts.ctypes.data, e, b,
                                       1 if on_dev else 0, _stream_ptr(stream))
    _check(rc, "jefi_eval_fields_multi")


def jefi_checkpoint(h: Handle, stream=None) -> bytes:
    """The handle's resident history as an opaque image (see jefi_restore)."""
    n = ctypes.c_size_t()
    _check(load().jefi_checkpoint_bytes(h.ptr, ctypes.byref(n)), "jefi_checkpoint_bytes")
    buf = ctypes.create_string_buffer(n.value)
    _check(load().jefi_checkpoint(h.ptr, ctypes.cast(buf, ctypes.c_void_p), n.value, _stream_ptr(stream)),
           "jefi_checkpoint")
    return buf.raw


def jefi_restore(h: Handle, image: bytes, stream=None):
    """Load a jefi_checkpoint image into a handle created with the same source
    grid and history parameters."""
    buf = ctypes.create_string_buffer(bytes(image), len(image))
    _check(load().jefi_restore(h.ptr, ctypes.cast(buf, ctypes.c_void_p), len(image), _stream_ptr(stream)),
           "jefi_restore")


def jefi_select_kernel(h: Handle, mode: int, t: float = 0.0, stream=None) -> int:
    """Choose the FP32 sum kernel of h (JEFI_KERNEL_MEASURE times both at t
    and keeps the faster; _DIRECT / _STAGED switch).  Returns the staged band
    in use, 0 for the direct gather."""
    band = ctypes.c_int32()
    rc = load().jefi_select_kernel(h.ptr, int(mode), float(t), ctypes.byref(band), _stream_ptr(stream))
    _check(rc, "jefi_select_kernel")
    return band.value


def jefi_valid_window(h: Handle):
    lo, hi = ctypes.c_double(), ctypes.c_double()
    rc = load().jefi_valid_window(h.ptr, ctypes.byref(lo), ctypes.byref(hi))
    _check(rc, "jefi_valid_window")
    return lo.value, hi.value


def jefi_get_info(h: Handle) -> dict:
    info = jefi_info()
    _check(load().jefi_get_info(h.ptr, ctypes.byref(info)), "jefi_get_info")
    return info.as_dict()


def jefi_reset_stats(h: Handle):
    _check(load().jefi_reset_stats(h.ptr), "jefi_reset_stats")


def jefi_debug_slots(h: Handle, t: float, stream=None) -> np.ndarray:
    out = np.empty((h.n_obs, h.n_src), dtype=np.int32)
    rc = load().jefi_debug_slots(h.ptr, float(t), out.ctypes.data, _stream_ptr(stream))
    _check(rc, "jefi_debug_slots")
    return out


def jefi_host_pair_slots(xo, xs, t, t0, c, dt) -> np.ndarray:
    xo = np.ascontiguousarray(xo, dtype=np.float64).reshape(-1, 3)
    xs = np.ascontiguousarray(xs, dtype=np.float64).reshape(-1, 3)
    out = np.empty(xo.shape[0], dtype=np.int64)
    load().jefi_host_pair_slots(xo.shape[0], xo.ctypes.data, xs.ctypes.data, float(t), float(t0),
                                float(c), float(dt), out.ctypes.data)
    return out


def jefi_host_split_plan(n_tiles: int, n_bricks: int, max_splits: int, times_per_launch: int,
                         resident_ctas: int):
    """(n_split, bricks_per_split, merge) of the library's split rule (host only)."""
    out = [ctypes.c_int32(0) for _ in range(3)]
    _check(load().jefi_host_split_plan(int(n_tiles), int(n_bricks), int(max_splits), int(times_per_launch),
                                       int(resident_ctas), *(ctypes.byref(o) for o in out)),
           "jefi_host_split_plan")
    return tuple(o.value for o in out)


def jefi_destroy(h: Handle):
    if h.ptr:
        rc = load().jefi_destroy(h.ptr)
        h.ptr = ctypes.c_void_p()
        _check(rc, "jefi_destroy")


# ---------------------------------------------------------------------------- conveniences
def eval_fields(h: Handle, t, stream=None):
    """E, B at time t (or times) as new torch CUDA tensors, FP64 [.., N_obs, 3]."""
    import torch

    if np.ndim(t) == 0:
        E = torch.empty((h.n_obs, 3), dtype=torch.float64, device="cuda")
        B = torch.empty_like(E)
        jefi_eval_fields(h, float(t), E, B, stream)
    else:
        ts = np.asarray(t, dtype=np.float64)
        E = torch.empty((ts.shape[0], h.n_obs, 3), dtype=torch.float64, device="cuda")
        B = torch.empty_like(E)
        jefi_eval_fields_multi(h, ts, E, B, stream)
    return E, B


def jefi_eval_fields_noalloc(src: jefi_grid, obs, rho, J, params: jefi_params, t: float, E, B,
                             stream=None):
    """FP64 fields at time t with no device allocation by the library.

    For callers that cannot allocate device memory at this point (see
    include/jefi.h): every buffer is the caller's own -- obs [N_obs, 3],
    rho [n_slices, N_src], J [n_slices, N_src, 3], E and B [N_obs, 3], all
    contiguous float64 CUDA tensors, N_src = src.n[0] * src.n[1] * src.n[2].
    The library cannot see the size of a device buffer, so the shapes are
    checked here, before anything reaches the GPU (ValueError otherwise).
    Returns after E and B are written on `stream`.
    """
    n_src = int(src.n[0]) * int(src.n[1]) * int(src.n[2])

    def shape(x):
        return tuple(int(d) for d in x.shape) if hasattr(x, "shape") else None

    if shape(obs) is None or len(shape(obs)) != 2 or shape(obs)[1] != 3:
        raise ValueError(f"obs must have shape (n_obs, 3), got {shape(obs)}")
    n_obs = shape(obs)[0]
    if shape(rho) is None or len(shape(rho)) != 2 or shape(rho)[1] != n_src:
        raise ValueError(f"rho must have shape (n_slices, {n_src}), got {shape(rho)}")
    n_slices = shape(rho)[0]
    if shape(J) != (n_slices, n_src, 3):
        raise ValueError(f"J must have shape {(n_slices, n_src, 3)}, got {shape(J)}")
    for name, x in (("E", E), ("B", B)):
        if shape(x) != (n_obs, 3):
            raise ValueError(f"{name} must have shape {(n_obs, 3)}, got {shape(x)}")
    bufs = [_buf(x) for x in (obs, rho, J, E, B)]
    if not all(b[1] for b in bufs):
        raise ValueError("jefi_eval_fields_noalloc takes device (CUDA) tensors only")
    rc = load().jefi_eval_fields_noalloc(ctypes.byref(src), bufs[0][0], n_obs, bufs[1][0], bufs[2][0],
                                         n_slices, ctypes.byref(params), float(t), bufs[3][0],
                                         bufs[4][0], _stream_ptr(stream))
    _check(rc, "jefi_eval_fields_noalloc")


def jefi_eval_batch(handles, times, E_list, B_list, stream=None):
    """Evaluate handles[i] at times[i] into E_list[i], B_list[i] (CUDA float64
    tensors [N_obs_i, 3]) in one batched launch."""
    n = len(handles)
    if not (len(times) == len(E_list) == len(B_list) == n):
        raise ValueError("handles, times and outputs must have the same length")
    hs = (ctypes.c_void_p * n)(*[h.ptr.value for h in handles])
    ts = (ctypes.c_double * n)(*[float(x) for x in times])
    es, bs = [], []
    for E, B in zip(E_list, B_list):
        e, on_e, _ = _buf(E)
        b, on_b, _ = _buf(B)
        if not (on_e and on_b):
            raise ValueError("jefi_eval_batch writes device (CUDA) tensors only")
        es.append(e)
        bs.append(b)
    ep = (ctypes.c_void_p * n)(*es)
    bp = (ctypes.c_void_p * n)(*bs)
    rc = load().jefi_eval_batch(hs, ts, ep, bp, n, _stream_ptr(stream))
    _check(rc, "jefi_eval_batch")


class BatchPlan:
    """Owns a jefi_batch_plan and keeps its handles and output tensors alive."""

    def __init__(self, ptr, handles, keep):
        self.ptr = ptr
        self.handles = handles
        self._keep = keep


def _times(plan: BatchPlan, times):
    n = len(plan.handles)
    if len(times) != n:
        raise ValueError("one time per batch entry")
    return (ctypes.c_double * max(n, 1))(*[float(x) for x in times])


def jefi_batch_plan_create(handles, E_list, B_list) -> BatchPlan:
    """Record the batched evaluation of handles[i] into E_list[i], B_list[i]
    (CUDA float64 tensors [N_obs_i, 3], fixed for the plan's life) as CUDA
    graphs (see include/jefi.h)."""
    n = len(handles)
    if not (len(E_list) == len(B_list) == n):
        raise ValueError("handles and outputs must have the same length")
    es, bs = [], []
    for E, B in zip(E_list, B_list):
        e, on_e, _ = _buf(E)
        b, on_b, _ = _buf(B)
        if not (on_e and on_b):
            raise ValueError("a batch plan writes device (CUDA) tensors only")
        es.append(e)
        bs.append(b)
    hs = (ctypes.c_void_p * max(n, 1))(*[h.ptr.value for h in handles])
    ep = (ctypes.c_void_p * max(n, 1))(*es)
    bp = (ctypes.c_void_p * max(n, 1))(*bs)
    out = ctypes.c_void_p()
    rc = load().jefi_batch_plan_create(hs, ep, bp, n, ctypes.byref(out))
    _check(rc, "jefi_batch_plan_create")
    return BatchPlan(out, list(handles), (list(E_list), list(B_list)))


def jefi_batch_plan_launch(plan: BatchPlan, times, stream=None):
    """Evaluate entry i at times[i]: one graph launch, asynchronous on `stream`."""
    rc = load().jefi_batch_plan_launch(plan.ptr, _times(plan, times), _stream_ptr(stream))
    _check(rc, "jefi_batch_plan_launch")


def jefi_batch_plan_tune(plan: BatchPlan, times, stream=None) -> dict:
    """Autotune the plan's kernels and source splits at `times`; returns the report."""
    rep = jefi_tune_report()
    rc = load().jefi_batch_plan_tune(plan.ptr, _times(plan, times), _stream_ptr(stream), ctypes.byref(rep))
    _check(rc, "jefi_batch_plan_tune")
    return rep.as_dict()


def jefi_batch_plan_destroy(plan: BatchPlan):
    if plan.ptr is not None and plan.ptr.value:
        rc = load().jefi_batch_plan_destroy(plan.ptr)
        _check(rc, "jefi_batch_plan_destroy")
        plan.ptr = None


def jefi_create_view(base: Handle, obs_grid: Optional[jefi_grid] = None, obs_points=None, stream=None):
    """Observation view over base's resident history (see include/jefi.h)."""
    keep = [base]
    pts_ptr, n_obs = None, 0
    if obs_grid is None:
        pts = np.ascontiguousarray(obs_points, dtype=np.float64).reshape(-1, 3)
        pts_ptr, n_obs = pts.ctypes.data, pts.shape[0]
        keep.append(pts)
    out = ctypes.c_void_p()
    rc = load().jefi_create_view(base.ptr, ctypes.byref(obs_grid) if obs_grid is not None else None,
                                 pts_ptr, n_obs, _stream_ptr(stream), ctypes.byref(out))
    _check(rc, "jefi_create_view")
    h = Handle(out, keep)
    info = jefi_get_info(h)
    h.n_obs = int(info["n_obs"])
    h.n_src = int(info["n_src"])
    return h


def jefi_debug_wait_timeout(limit_s: float, stream=None) -> int:
    """Status of a bounded device wait that nothing completes (JEFI_ETIMEOUT expected)."""
    return int(load().jefi_debug_wait_timeout(float(limit_s), _stream_ptr(stream)))
