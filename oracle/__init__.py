"""FP64 CPU oracle for batched Bezier / chain / B-spline / NURBS / surface /
volume evaluation, its gradients and the fused polyline length.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
library (``paper_2603_15447_gb300``) never imports it, and the two share no
code: the C source here (``oracle.c``) is compiled with the host C compiler
into ``liboracle.so`` and reached through ctypes.

Every function takes NumPy arrays; FP32 inputs are widened to FP64 exactly,
so the oracle sees bit-for-bit the values a GPU kernel sees.  Work is split
over curves across host threads (ctypes releases the GIL for the duration of
each foreign call), which is how the CPU baseline uses all host cores.

What each function computes, and the passage of the paper it follows, is
stated in ``oracle.c``.  Parity status: every function here is pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_*.py`` (exact rational
arithmetic, library routines, closed forms and invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.c_int64
_INT = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with the host C compiler."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-ffp-contract=off",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.orc_grid_value.restype = ctypes.c_double
            lib.orc_grid_value.argtypes = [_I64, _I64]
            lib.orc_bezier.argtypes = [_D, _D, _I64, _INT, _INT, _D, _I64, _I64, _D]
            lib.orc_bezier_grid.argtypes = [_D, _D, _I64, _INT, _INT, _I64, _D]
            lib.orc_chain.argtypes = [_D, _I64, _INT, _INT, _INT, _D, _I64, _I64, _D]
            lib.orc_clamped_uniform_knots.argtypes = [_INT, _INT, _D]
            lib.orc_bspline.argtypes = [_D, _D, _D, _I64, _INT, _INT, _INT, _D, _I64, _I64, _D]
            lib.orc_surface.argtypes = [_D, _I64, _INT, _INT, _INT, _INT, _INT, _D]
            lib.orc_volume.argtypes = [_D, _I64, _INT, _INT, _INT, _INT, _INT, _INT, _INT, _D]
            lib.orc_bezier_grad.argtypes = [_D, _D, _I64, _INT, _INT, _D, _I64, _I64, _D, _D, _D, _D]
            lib.orc_polyline_length.argtypes = [_D, _I64, _I64, _INT, _D]
            lib.orc_lowbias32.restype = ctypes.c_uint32
            lib.orc_lowbias32.argtypes = [ctypes.c_uint32]
            lib.orc_stream_key.restype = ctypes.c_uint32
            lib.orc_stream_key.argtypes = [ctypes.c_uint64, ctypes.c_uint32]
            lib.orc_hash_t.argtypes = [ctypes.c_uint64, ctypes.c_uint32, _I64, _I64, _I64, _D]
            _lib = lib
    return _lib


def _f64(a):
    return None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a):
    return None if a is None else a.ctypes.data_as(_D)


def default_threads() -> int:
    return int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))


def _chunks(n: int, threads: int):
    threads = max(1, min(threads, n))
    step = (n + threads - 1) // threads
    return [(s, min(n, s + step)) for s in range(0, n, step)]


def _parallel(n_items, threads, fn):
    parts = _chunks(n_items, threads)
    if len(parts) <= 1:
        for s, e in parts:
            fn(s, e)
        return
    with ThreadPoolExecutor(len(parts)) as ex:
        list(ex.map(lambda se: fn(*se), parts))


def _t_layout(t, n_curves):
    """Return (t as FP64 [n_curves or 1][n_t], stride)."""
    t = _f64(t)
    if t.ndim == 1:
        return t.reshape(1, -1), 0
    assert t.shape[0] == n_curves
    return t, t.shape[1]


# ---------------------------------------------------------------- curves

def bezier(ctrl, t, weights=None, threads=None):
    """Bernstein-sum Bezier (rational if weights given).

    ctrl [B][d+1][dim]; t [n_t] shared or [B][n_t]; weights [B][d+1].
    Returns FP64 [B][n_t][dim]."""
    lib = _load()
    ctrl = _f64(ctrl)
    B, d1, dim = ctrl.shape
    w = _f64(weights)
    tt, stride = _t_layout(t, B)
    n_t = tt.shape[1]
    out = np.empty((B, n_t, dim), np.float64)

    def run(s, e):
        lib.orc_bezier(_p(ctrl[s:e]), _p(w[s:e]) if w is not None else None, e - s, d1 - 1, dim,
                       _p(tt[s:e] if stride else tt), stride, n_t, _p(out[s:e]))

    _parallel(B, threads or default_threads(), run)
    return out


def bezier_grid(ctrl, n_t, weights=None, threads=None):
    """Bezier curves on the uniform grid t_j = fl32(j)/fl32(n_t-1)."""
    lib = _load()
    ctrl = _f64(ctrl)
    B, d1, dim = ctrl.shape
    w = _f64(weights)
    out = np.empty((B, n_t, dim), np.float64)

    def run(s, e):
        lib.orc_bezier_grid(_p(ctrl[s:e]), _p(w[s:e]) if w is not None else None, e - s, d1 - 1, dim,
                            n_t, _p(out[s:e]))

    _parallel(B, threads or default_threads(), run)
    return out


def grid(n):
    """The FP32 uniform grid values a/(n-1) as FP64."""
    lib = _load()
    return np.array([lib.orc_grid_value(a, n) for a in range(n)], np.float64)


def chain(ctrl, n_seg, degree, t, threads=None):
    """C0 piecewise Bezier chain; ctrl [C][n_seg*degree+1][dim], t in [0, n_seg]."""
    lib = _load()
    ctrl = _f64(ctrl)
    C, npts, dim = ctrl.shape
    assert npts == n_seg * degree + 1
    tt, stride = _t_layout(t, C)
    n_t = tt.shape[1]
    out = np.empty((C, n_t, dim), np.float64)

    def run(s, e):
        lib.orc_chain(_p(ctrl[s:e]), e - s, n_seg, degree, dim, _p(tt[s:e] if stride else tt), stride,
                      n_t, _p(out[s:e]))

    _parallel(C, threads or default_threads(), run)
    return out


def clamped_uniform_knots(n_ctrl, degree):
    lib = _load()
    U = np.empty(n_ctrl + degree + 1, np.float64)
    lib.orc_clamped_uniform_knots(n_ctrl, degree, _p(U))
    return U


def bspline(ctrl, degree, t, weights=None, knots=None, threads=None):
    """Cox-de Boor B-spline / NURBS; ctrl [B][n][dim]; knots [B][n+p+1] or None
    (clamped uniform); weights [B][n] or None (integral)."""
    lib = _load()
    ctrl = _f64(ctrl)
    B, n, dim = ctrl.shape
    w = _f64(weights)
    U = _f64(knots)
    tt, stride = _t_layout(t, B)
    n_t = tt.shape[1]
    out = np.empty((B, n_t, dim), np.float64)

    def run(s, e):
        lib.orc_bspline(_p(ctrl[s:e]), _p(w[s:e]) if w is not None else None,
                        _p(U[s:e]) if U is not None else None, e - s, n, degree, dim,
                        _p(tt[s:e] if stride else tt), stride, n_t, _p(out[s:e]))

    _parallel(B, threads or default_threads(), run)
    return out


# ---------------------------------------------------------------- tensor products

def surface(ctrl, nu, nv, threads=None):
    """ctrl [n][du+1][dv+1][dim] -> [n][nu][nv][dim] on uniform grids."""
    lib = _load()
    ctrl = _f64(ctrl)
    n, du1, dv1, dim = ctrl.shape
    out = np.empty((n, nu, nv, dim), np.float64)

    def run(s, e):
        lib.orc_surface(_p(ctrl[s:e]), e - s, du1 - 1, dv1 - 1, dim, nu, nv, _p(out[s:e]))

    _parallel(n, threads or default_threads(), run)
    return out


def volume(ctrl, nu, nv, nw, threads=None):
    """ctrl [n][du+1][dv+1][dw+1][dim] -> [n][nu][nv][nw][dim]."""
    lib = _load()
    ctrl = _f64(ctrl)
    n, du1, dv1, dw1, dim = ctrl.shape
    out = np.empty((n, nu, nv, nw, dim), np.float64)

    def run(s, e):
        lib.orc_volume(_p(ctrl[s:e]), e - s, du1 - 1, dv1 - 1, dw1 - 1, dim, nu, nv, nw, _p(out[s:e]))

    _parallel(n, threads or default_threads(), run)
    return out


# ---------------------------------------------------------------- gradients

def bezier_grad(ctrl, t, grad_out, weights=None, threads=None):
    """Analytic gradients of the (rational) Bezier curve.

    Returns (grad_ctrl [B][d+1][dim], grad_w [B][d+1] or None,
    grad_t [B][n_t] for per-curve t, or [n_t] summed over curves for shared t)."""
    lib = _load()
    ctrl = _f64(ctrl)
    B, d1, dim = ctrl.shape
    w = _f64(weights)
    g = _f64(grad_out)
    tt, stride = _t_layout(t, B)
    n_t = tt.shape[1]
    gc = np.empty((B, d1, dim), np.float64)
    gw = np.empty((B, d1), np.float64) if w is not None else None
    if stride:
        gt = np.empty((B, n_t), np.float64)

        def run(s, e):
            lib.orc_bezier_grad(_p(ctrl[s:e]), _p(w[s:e]) if w is not None else None, e - s, d1 - 1, dim,
                                _p(tt[s:e]), stride, n_t, _p(g[s:e]), _p(gc[s:e]),
                                _p(gw[s:e]) if gw is not None else None, _p(gt[s:e]))

        _parallel(B, threads or default_threads(), run)
    else:
        parts = _chunks(B, threads or default_threads())
        partial = np.zeros((len(parts), n_t), np.float64)

        def run2(i):
            s, e = parts[i]
            lib.orc_bezier_grad(_p(ctrl[s:e]), _p(w[s:e]) if w is not None else None, e - s, d1 - 1, dim,
                                _p(tt), 0, n_t, _p(g[s:e]), _p(gc[s:e]),
                                _p(gw[s:e]) if gw is not None else None, _p(partial[i]))

        with ThreadPoolExecutor(len(parts)) as ex:
            list(ex.map(run2, range(len(parts))))
        gt = partial.sum(axis=0)
    return gc, gw, gt


# ---------------------------------------------------------------- polyline length

def polyline_length(points):
    """points [n][n_pts][dim] -> [n] sum of segment lengths in index order."""
    lib = _load()
    pts = _f64(points)
    n, n_pts, dim = pts.shape
    out = np.empty(n, np.float64)
    lib.orc_polyline_length(_p(pts), n, n_pts, dim, _p(out))
    return out


# ---------------------------------------------------------------- counter hash

def lowbias32(x: int) -> int:
    return int(_load().orc_lowbias32(ctypes.c_uint32(x & 0xFFFFFFFF)))


def stream_key(seed: int, stream: int) -> int:
    return int(_load().orc_stream_key(ctypes.c_uint64(seed & (2**64 - 1)), ctypes.c_uint32(stream)))


def hash_t(seed: int, stream: int, c0: int, n_curves: int, n_t: int):
    """Parameters a kernel draws in-kernel: [n_curves][n_t] FP64 holding FP32 values."""
    lib = _load()
    t = np.empty((n_curves, n_t), np.float64)
    lib.orc_hash_t(ctypes.c_uint64(seed & (2**64 - 1)), ctypes.c_uint32(stream), c0, n_curves, n_t, _p(t))
    return t


def hashed_bezier_polyline_length(ctrl, n_t, seed, stream, c0=0, threads=None):
    """Polyline length of each Bezier curve sampled at its in-kernel hash
    parameters (the fused evaluate-and-reduce workload): for every curve the
    oracle draws t, evaluates the Bernstein sum and sums segment lengths."""
    ctrl = _f64(ctrl)
    B = ctrl.shape[0]
    out = np.empty(B, np.float64)

    def run(s, e):
        t = hash_t(seed, stream, c0 + s, e - s, n_t)
        pts = bezier(ctrl[s:e], t, threads=1)
        out[s:e] = polyline_length(pts)

    _parallel(B, threads or default_threads(), run)
    return out
