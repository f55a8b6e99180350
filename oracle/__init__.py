"""FP64 CPU oracle for the discretised Jefimenko sum (paper Sec. 2.2, Eqs. E-1, B-1, tr-1).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this package.  The GPU library
never imports, links or calls it; the two share no code.

The arithmetic lives in ``jefi_oracle.c`` (plain C, FP64, Neumaier-compensated
sums, OpenMP over observation points).  This module builds it with gcc and
exposes thin numpy wrappers.  ``closed_forms`` holds the analytic fields the
oracle is pinned against.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jefi_oracle.c")
# JEFI_ORACLE_LIB: load a prebuilt oracle library instead (the mutation test
# plants mistakes in a copy of jefi_oracle.c and runs the pins against it).
_LIB_OVERRIDE = os.environ.get("JEFI_ORACLE_LIB")
_LIB_PATH = _LIB_OVERRIDE or os.path.join(_HERE, "libjefi_oracle.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off: no fused multiply-add anywhere (gcc contracts by default
# on aarch64), so every product and sum is rounded as written.
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-std=c11"]

ENOTYET = 3


def build(force: bool = False) -> str:
    """Compile the oracle shared library in-tree and return its path."""
    if _LIB_OVERRIDE:
        return _LIB_PATH
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            D = ctypes.c_double
            lib.oracle_fields.restype = ctypes.c_int
            lib.oracle_fields.argtypes = [P, P, P, I64, P, I64, P, P, P, P,
                                          D, D, D, D, D, P, D, P, P, P, P, P, ctypes.c_int]
            lib.oracle_fields_interp.restype = ctypes.c_int
            lib.oracle_fields_interp.argtypes = [P, P, P, I64, P, I64, P, P, P, P,
                                                 D, D, D, D, D, P, D, P, P, ctypes.c_int]
            lib.oracle_all_slots.restype = None
            lib.oracle_all_slots.argtypes = [P, P, P, I64, P, D, D, D, P, D, P, ctypes.c_int]
            lib.oracle_pair_slots.restype = None
            lib.oracle_pair_slots.argtypes = [I64, P, P, D, D, D, D, P]
            lib.oracle_cell_center.restype = D
            lib.oracle_cell_center.argtypes = [D, D, I64]
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def cell_centers(n: int, lo: float, d: float) -> np.ndarray:
    """Cell centres lo + (i + 0.5) d, rounded exactly as the oracle rounds them."""
    lib = _load()
    return np.array([lib.oracle_cell_center(float(lo), float(d), i) for i in range(int(n))])


def fields(src_n, src_lo, src_d, obs, rho, J, *, c=1.0, k_e=1.0, k_b=1.0, dt, t0=0.0,
           screen=None, t, drho=None, dJ=None, threads=0, with_abs=False, with_slots=False):
    """E and B at time ``t`` for every point of ``obs`` ([n_obs, 3]).

    ``rho`` is [n_slices, Ns] and ``J`` [n_slices, Ns, 3]; slice n holds the
    sources at t0 + n dt and the cell index runs x fastest.  ``screen`` is the
    per-axis screening half-width (default: half the source cell).  Supplying
    ``drho``/``dJ`` replaces the backward difference.  Raises ``ValueError``
    when a pair needs a slice that is not in the history.
    """
    lib = _load()
    src_n = np.ascontiguousarray(src_n, dtype=np.int32).reshape(3)
    src_lo = _f64(src_lo, (3,))
    src_d = _f64(src_d, (3,))
    obs = _f64(obs, (-1, 3))
    Ns = int(np.prod(src_n))
    rho = _f64(rho, (-1, Ns))
    n_slices = rho.shape[0]
    J = _f64(J, (n_slices, Ns, 3))
    if drho is not None:
        drho = _f64(drho, (n_slices, Ns))
    if dJ is not None:
        dJ = _f64(dJ, (n_slices, Ns, 3))
    if screen is None:
        screen = src_d / 2.0
    screen = _f64(screen, (3,))
    n_obs = obs.shape[0]
    E = np.zeros((n_obs, 3))
    B = np.zeros((n_obs, 3))
    aE = np.zeros((n_obs, 3)) if with_abs else None
    aB = np.zeros((n_obs, 3)) if with_abs else None
    sr = np.zeros(2, dtype=np.int64)
    rc = lib.oracle_fields(_ptr(src_n), _ptr(src_lo), _ptr(src_d), n_obs, _ptr(obs),
                           n_slices, _ptr(rho), _ptr(J), _ptr(drho), _ptr(dJ),
                           float(c), float(k_e), float(k_b), float(dt), float(t0),
                           _ptr(screen), float(t), _ptr(E), _ptr(B), _ptr(aE), _ptr(aB),
                           _ptr(sr), int(threads))
    if rc == ENOTYET:
        raise ValueError("oracle: time t needs a slice beyond the history")
    if rc != 0:
        raise ValueError(f"oracle: invalid arguments (code {rc})")
    out = [E, B]
    if with_abs:
        out += [aE, aB]
    if with_slots:
        out.append((int(sr[0]), int(sr[1])))
    return tuple(out)


def fields_interp(src_n, src_lo, src_d, obs, rho, J, *, c=1.0, k_e=1.0, k_b=1.0, dt, t0=0.0,
                  screen=None, t, drho=None, dJ=None, threads=0):
    """Second-order variant of ``fields``: sources linearly interpolated
    between slices n and n+1 at the retarded time, derivatives supplied or
    central differences (f[k+1] - f[k-1]) / (2 dt), both interpolated; slices
    before the first are zero.  Needs slices up to n+1 (supplied) or n+2
    (central); raises ``ValueError`` otherwise.
    """
    lib = _load()
    src_n = np.ascontiguousarray(src_n, dtype=np.int32).reshape(3)
    src_lo = _f64(src_lo, (3,))
    src_d = _f64(src_d, (3,))
    obs = _f64(obs, (-1, 3))
    Ns = int(np.prod(src_n))
    rho = _f64(rho, (-1, Ns))
    n_slices = rho.shape[0]
    J = _f64(J, (n_slices, Ns, 3))
    if (drho is None) != (dJ is None):
        raise ValueError("supply both drho and dJ, or neither")
    if drho is not None:
        drho = _f64(drho, (n_slices, Ns))
        dJ = _f64(dJ, (n_slices, Ns, 3))
    if screen is None:
        screen = src_d / 2.0
    screen = _f64(screen, (3,))
    n_obs = obs.shape[0]
    E = np.zeros((n_obs, 3))
    B = np.zeros((n_obs, 3))
    rc = lib.oracle_fields_interp(_ptr(src_n), _ptr(src_lo), _ptr(src_d), n_obs, _ptr(obs),
                                  n_slices, _ptr(rho), _ptr(J), _ptr(drho), _ptr(dJ),
                                  float(c), float(k_e), float(k_b), float(dt), float(t0),
                                  _ptr(screen), float(t), _ptr(E), _ptr(B), int(threads))
    if rc == ENOTYET:
        raise ValueError("oracle: time t needs a slice beyond the history")
    if rc != 0:
        raise ValueError(f"oracle: invalid arguments (code {rc})")
    return E, B


def all_slots(src_n, src_lo, src_d, obs, *, c=1.0, dt, t0=0.0, screen=None, t, threads=0):
    """Slot of every (observation point, source cell) pair, [n_obs, Ns] int64.

    Screened pairs are reported as the minimum int64.
    """
    lib = _load()
    src_n = np.ascontiguousarray(src_n, dtype=np.int32).reshape(3)
    src_lo = _f64(src_lo, (3,))
    src_d = _f64(src_d, (3,))
    obs = _f64(obs, (-1, 3))
    if screen is None:
        screen = src_d / 2.0
    screen = _f64(screen, (3,))
    out = np.empty((obs.shape[0], int(np.prod(src_n))), dtype=np.int64)
    lib.oracle_all_slots(_ptr(src_n), _ptr(src_lo), _ptr(src_d), obs.shape[0], _ptr(obs),
                         float(c), float(dt), float(t0), _ptr(screen), float(t), _ptr(out),
                         int(threads))
    return out


def pair_slots(xo, xs, *, t, t0=0.0, c=1.0, dt):
    """Slots of explicit pairs (xo[k], xs[k]), int64 array."""
    lib = _load()
    xo = _f64(xo, (-1, 3))
    xs = _f64(xs, (-1, 3))
    out = np.empty(xo.shape[0], dtype=np.int64)
    lib.oracle_pair_slots(xo.shape[0], _ptr(xo), _ptr(xs), float(t), float(t0), float(c),
                          float(dt), _ptr(out))
    return out


SCREENED = np.iinfo(np.int64).min
