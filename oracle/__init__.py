"""CPU oracle for the moco translation search (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package. The product library never does, and this package
never imports the product: the two share only the seeded input generator.

``moco_oracle.c`` states the method of Section 2 as a brute force in exact
int64 (FP64 for the real-valued soft-min form). This module compiles it with
gcc into ``oracle/_build/liboracle.so`` and exposes numpy wrappers.

Parity pins: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` against closed forms, invariants, library
routines (scipy correlation, numpy FFT following the paper's zero-padding
recipe) and finite differences. The 50-step template refinement built on the
gradient is parity unpinned beyond its first gradient.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "moco_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP); returns the shared-library path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            L.oracle_area.restype = i64
            L.oracle_area.argtypes = [i32, i32, i32, i32]
            L.oracle_ssd_one.restype = i64
            L.oracle_ssd_one.argtypes = [P, P, i32, i32, i32, i32]
            L.oracle_ssd_all.restype = None
            L.oracle_ssd_all.argtypes = [P, P, i32, i32, i32, P]
            L.oracle_downsample.restype = None
            L.oracle_downsample.argtypes = [P, i32, i32, P]
            L.oracle_levels.restype = i32
            L.oracle_levels.argtypes = [i32, i32]
            L.oracle_align.restype = i32
            L.oracle_align.argtypes = [P, i64, P, i32, i32, i32, i32, P, P, P, P, P, i32]
            L.oracle_cost_surface.restype = i32
            L.oracle_cost_surface.argtypes = [P, i64, P, i32, i32, i32, i32, P, P, i32]
            L.oracle_cost_f64.restype = None
            L.oracle_cost_f64.argtypes = [P, P, i32, i32, i32, P]
            L.oracle_median.restype = dbl
            L.oracle_median.argtypes = [P, i32]
            L.oracle_softmin_loss.restype = dbl
            L.oracle_softmin_loss.argtypes = [P, i64, P, i32, i32, i32, P, P, P, P, i32]
            L.oracle_refine.restype = i32
            L.oracle_refine.argtypes = [P, i64, P, i32, i32, P, P, P, i32]
            L.oracle_apply_shifts.restype = None
            L.oracle_apply_shifts.argtypes = [P, i64, i32, i32, P, ctypes.c_uint16, P, P]
            _lib = L
    return _lib


def _p(x):
    return x.ctypes.data_as(ctypes.c_void_p) if x is not None else None


def _c(x, dtype):
    return np.ascontiguousarray(x, dtype=dtype)


def area(m, n, s, t) -> int:
    return int(lib().oracle_area(m, n, s, t))


def levels(m, n) -> int:
    return int(lib().oracle_levels(m, n))


def ssd_all(a, b, w) -> np.ndarray:
    """Exact int64 Area*f for every shift: array (2w-1, 2w-1) indexed [s+w-1, t+w-1]."""
    a = _c(a, np.int32); b = _c(b, np.int32)
    m, n = a.shape
    W = 2 * w - 1
    S = np.empty((W, W), np.int64)
    lib().oracle_ssd_all(_p(a), _p(b), m, n, w, _p(S))
    return S


def downsample(a) -> np.ndarray:
    a = _c(a, np.uint16)
    m, n = a.shape
    out = np.empty((m // 2, n // 2), np.int32)
    lib().oracle_downsample(_p(a), m, n, _p(out))
    return out


def align(frames, template, w, levels=-1, nthreads=0):
    """Exhaustive search + upsampling jitter. levels: -1 the paper's rule (one
    level above 256x256), else 0..4 (the search on level L, then one 3x3
    refinement per level down to full resolution). Returns a dict of numpy
    arrays: shifts (T,2), coarse (T,2) on the searched level, fbest (T,),
    margin (T,), ffinal (T,) at full resolution."""
    frames = _c(frames, np.uint16)
    template = _c(template, np.uint16)
    if frames.ndim == 2:
        frames = frames[None]
    T, m, n = frames.shape
    out = dict(shifts=np.empty((T, 2), np.int32), coarse=np.empty((T, 2), np.int32),
               fbest=np.empty(T), margin=np.empty(T), ffinal=np.empty(T))
    rc = lib().oracle_align(_p(frames), T, _p(template), m, n, w, levels, _p(out["shifts"]),
                            _p(out["coarse"]), _p(out["fbest"]), _p(out["margin"]),
                            _p(out["ffinal"]), nthreads)
    if rc != 0:
        raise ValueError("oracle_align rejected the arguments (rc=%d)" % rc)
    return out


def refine(frames, template, coarse, nthreads=0):
    """The upsampling step alone: the best of the nine full-resolution shifts
    around 2 * coarse per frame. Returns (shifts (T,2), ffinal (T,)); a frame
    whose coarse shift leaves a candidate without overlap gets INT32_MIN."""
    frames = _c(frames, np.uint16)
    template = _c(template, np.uint16)
    if frames.ndim == 2:
        frames = frames[None]
    T, m, n = frames.shape
    coarse = _c(coarse, np.int32).reshape(T, 2)
    shifts = np.empty((T, 2), np.int32)
    ffinal = np.empty(T)
    rc = lib().oracle_refine(_p(frames), T, _p(template), m, n, _p(coarse), _p(shifts), _p(ffinal), nthreads)
    if rc != 0:
        raise MemoryError("oracle_refine failed (rc=%d)" % rc)
    return shifts, ffinal


def cost_surface(frames, template, w, levels=-1, with_sums=False, nthreads=0):
    """FP64 cost surface (T, 2w-1, 2w-1) in box-mean units (and exact sums)."""
    frames = _c(frames, np.uint16)
    template = _c(template, np.uint16)
    if frames.ndim == 2:
        frames = frames[None]
    T, m, n = frames.shape
    W = 2 * w - 1
    cost = np.empty((T, W, W))
    S = np.empty((T, W, W), np.int64) if with_sums else None
    rc = lib().oracle_cost_surface(_p(frames), T, _p(template), m, n, w, levels, _p(cost),
                                   _p(S), nthreads)
    if rc != 0:
        raise ValueError("oracle_cost_surface rejected the arguments (rc=%d)" % rc)
    return (cost, S) if with_sums else cost


def cost_f64(a, b, w) -> np.ndarray:
    a = _c(a, np.float64); b = _c(b, np.float64)
    m, n = a.shape
    W = 2 * w - 1
    cost = np.empty((W, W))
    lib().oracle_cost_f64(_p(a), _p(b), m, n, w, _p(cost))
    return cost


def median(values) -> float:
    v = _c(values, np.float64).ravel()
    return float(lib().oracle_median(_p(v), v.size))


def softmin_tau(frames, template, w, scale=0.05):
    """Per-frame temperature: scale * median of the frame's cost surface."""
    frames = _c(frames, np.float64)
    if frames.ndim == 2:
        frames = frames[None]
    return np.array([scale * median(cost_f64(fr, template, w)) for fr in frames])


def softmin_loss(frames, template, w, tau, grad_template=False, grad_frames=False, nthreads=0):
    """Soft-min loss (FP64) with optional analytic gradients.
    Returns (loss, per_frame_loss, grad_template or None, grad_frames or None)."""
    frames = _c(frames, np.float64)
    template = _c(template, np.float64)
    if frames.ndim == 2:
        frames = frames[None]
    T, m, n = frames.shape
    tau = _c(tau, np.float64)
    lf = np.empty(T)
    gb = np.empty((m, n)) if grad_template else None
    ga = np.empty((T, m, n)) if grad_frames else None
    L = lib().oracle_softmin_loss(_p(frames), T, _p(template), m, n, w, _p(tau), _p(lf), _p(gb),
                                  _p(ga), nthreads)
    return float(L), lf, gb, ga


def apply_shifts(frames, shifts, fill=0, corrected=True, mean=True):
    """Corrected frames (T, m, n) uint16 and the corrected mean image (m, n)
    FP64 (see moco_oracle.c); returns (corrected or None, mean or None)."""
    frames = _c(frames, np.uint16)
    if frames.ndim == 2:
        frames = frames[None]
    T, m, n = frames.shape
    shifts = _c(shifts, np.int32).reshape(T, 2)
    out = np.empty((T, m, n), np.uint16) if corrected else None
    mu = np.empty((m, n)) if mean else None
    lib().oracle_apply_shifts(_p(frames), T, m, n, _p(shifts), int(fill), _p(out), _p(mu))
    return out, mu
