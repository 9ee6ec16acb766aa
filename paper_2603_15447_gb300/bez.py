"""Thin ctypes binding of libbez.so (C ABI in include/bez.h).

Argument marshalling only: every step of evaluation runs in the library's
CUDA kernels.  Arrays are torch tensors (CUDA or CPU; CPU tensors are staged
by the library itself) or NumPy arrays (host).  The binding never falls back
to a CPU implementation: if libbez.so is missing or no CUDA device is
present, calls raise.
"""
from __future__ import annotations

import ctypes
import enum
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbez.so")


class Status(enum.IntEnum):
    OK = 0
    INVALID_ARG = 1
    UNSUPPORTED = 2
    CUDA = 3
    OOM = 4
    TIMEOUT = 5


class Variant(enum.IntEnum):
    AUTO = 0
    HORNER = 1
    HORNER_CENTRED = 2
    BERNSTEIN = 3
    DECASTELJAU = 4
    SEILER = 5
    TEX_DECASTELJAU = 6
    TEX_SEILER = 7
    TEX_HYBRID = 8
    TENSOR = 9
    COISSUE = 10
    HALF2 = 11


class DType(enum.IntEnum):
    F32 = 0
    F16 = 1
    BF16 = 2


class OutMode(enum.IntEnum):
    POINTS = 0
    POLYLINE_LENGTH = 1


class TMode(enum.IntEnum):
    SHARED = 0
    PER_CURVE = 1
    UNIFORM = 2
    HASH = 3


class TexFormat(enum.IntEnum):
    AUTO = 0
    UNORM16 = 1
    UNORM8 = 2


class Opts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("dtype", ctypes.c_int32), ("out_mode", ctypes.c_int32),
                ("t_mode", ctypes.c_int32), ("seed", ctypes.c_uint64), ("stream_id", ctypes.c_uint32),
                ("sync", ctypes.c_int32), ("err_word", ctypes.c_void_p), ("tex_share", ctypes.c_int32),
                ("tex_format", ctypes.c_int32), ("tex_spread", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("timed_launches", ctypes.c_int64), ("timed_ms", ctypes.c_double)]


class BezError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{Status(status).name}: {msg}")
        self.status = Status(status)


_lib = None
_lib_lock = threading.Lock()
_VP, _I64, _INT = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int


def lib():
    """Load libbez.so (raises if it has not been built)."""
    global _lib
    with _lib_lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libbez.so not found at {LIB_PATH}: build it with "
                                   "`python -m paper_2603_15447_gb300.build` (needs nvcc)")
            L = ctypes.CDLL(LIB_PATH)
            L.bez_version.restype = ctypes.c_char_p
            L.bez_last_error.restype = ctypes.c_char_p
            L.bez_create.argtypes = [ctypes.POINTER(_VP), _INT]
            L.bez_destroy.argtypes = [_VP]
            L.bez_set_timing.argtypes = [_VP, _INT]
            L.bez_get_stats.argtypes = [_VP, ctypes.POINTER(Stats)]
            L.bez_reset_stats.argtypes = [_VP]
            L.bez_eval.argtypes = [_VP, _VP, _I64, _INT, _INT, _VP, _I64, _VP, ctypes.POINTER(Opts), _VP]
            L.bez_probe_filter.argtypes = [_VP, _VP, _I64, _VP, _VP]
            L.bez_probe_filter_2d.argtypes = [_VP, _VP, _I64, _VP, _VP]
            L.bez_eval_bspline.argtypes = [_VP, _VP, _VP, _I64, _INT, _INT, _INT, _VP, _I64, _VP,
                                           ctypes.POINTER(Opts), _VP]
            L.bez_eval_nurbs.argtypes = [_VP, _VP, _VP, _VP, _I64, _INT, _INT, _INT, _VP, _I64, _VP,
                                         ctypes.POINTER(Opts), _VP]
            L.bez_eval_surface.argtypes = [_VP, _VP, _I64, _INT, _INT, _INT, _INT, _INT, _VP, ctypes.POINTER(Opts),
                                           _VP]
            L.bez_eval_volume.argtypes = [_VP, _VP, _I64, _INT, _INT, _INT, _INT, _INT, _INT, _INT, _VP,
                                          ctypes.POINTER(Opts), _VP]
            L.bez_eval_backward.argtypes = [_VP, _VP, _VP, _I64, _INT, _INT, _VP, _I64, _VP, _VP, _VP, _VP,
                                            ctypes.POINTER(Opts), _VP]
            L.bez_eval_spline_noalloc.argtypes = [_VP, _VP, _VP, _I64, _INT, _INT, _INT, _VP, _I64, _VP,
                                                  ctypes.POINTER(Opts), _VP]
            L.bez_eval_piecewise.argtypes = [_VP, _VP, _I64, _INT, _INT, _INT, _VP, _I64, _VP, ctypes.POINTER(Opts),
                                             _VP]
            for name in ("bez_create", "bez_destroy", "bez_set_timing", "bez_get_stats", "bez_reset_stats",
                         "bez_eval", "bez_probe_filter", "bez_probe_filter_2d", "bez_eval_piecewise",
                         "bez_eval_bspline", "bez_eval_nurbs",
                         "bez_eval_spline_noalloc", "bez_eval_surface", "bez_eval_volume",
                         "bez_eval_backward"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def _check(st):
    if st != 0:
        raise BezError(st, lib().bez_last_error().decode())


# ---------------------------------------------------------------- marshalling

def _torch():
    import torch
    return torch


def _ptr(x):
    """Raw address of a contiguous torch tensor / NumPy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous, "arrays must be C-contiguous"
        return x.ctypes.data
    assert x.is_contiguous(), "tensors must be contiguous"
    return x.data_ptr()


def _is_cuda(x):
    return x is not None and not isinstance(x, np.ndarray) and x.is_cuda


def _stream_handle(stream, device):
    torch = _torch()
    if stream is None:
        return torch.cuda.current_stream(device).cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dtype_code(x):
    if isinstance(x, np.ndarray):
        m = {np.dtype(np.float32): DType.F32, np.dtype(np.float16): DType.F16}
        return m[x.dtype]
    torch = _torch()
    m = {torch.float32: DType.F32, torch.float16: DType.F16, torch.bfloat16: DType.BF16}
    if x.dtype not in m:
        raise TypeError(f"control points must be float32/float16/bfloat16, got {x.dtype}")
    return m[x.dtype]


def _empty_like_location(ref, shape):
    torch = _torch()
    if isinstance(ref, np.ndarray):
        return np.empty(shape, np.float32)
    return torch.empty(shape, dtype=torch.float32, device=ref.device)


class Context:
    """A libbez context on one CUDA device."""

    def __init__(self, device: int = 0):
        self.device = device
        h = _VP()
        _check(lib().bez_create(ctypes.byref(h), device))
        self.handle = h

    def close(self):
        if self.handle:
            lib().bez_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_timing(self, on: bool):
        _check(lib().bez_set_timing(self.handle, int(on)))

    def stats(self) -> dict:
        s = Stats()
        _check(lib().bez_get_stats(self.handle, ctypes.byref(s)))
        return {"launches": s.launches, "timed_launches": s.timed_launches, "timed_ms": s.timed_ms}

    def reset_stats(self):
        _check(lib().bez_reset_stats(self.handle))


_contexts: dict[int, Context] = {}


def context(device: int | None = None) -> Context:
    if device is None:
        device = _torch().cuda.current_device()
    if device not in _contexts:
        _contexts[device] = Context(device)
    return _contexts[device]


def _opts(variant, dtype, out_mode, t_mode, seed, stream_id, sync, tex_share=0, tex_format=TexFormat.AUTO,
          tex_spread=0):
    return Opts(int(variant), int(dtype), int(out_mode), int(t_mode), int(seed) & (2 ** 64 - 1),
                int(stream_id) & 0xFFFFFFFF, int(sync), None, int(tex_share), int(tex_format), int(tex_spread))


# ---------------------------------------------------------------- entry points

def bez_eval(ctrl, t=None, *, n_t=None, variant=Variant.AUTO, out_mode=OutMode.POINTS, t_mode=None,
             seed=0, stream_id=0, out=None, stream=None, sync=False, ctx=None, tex_share=0,
             tex_format=TexFormat.AUTO, tex_spread=0):
    """Evaluate Bezier curves ``ctrl`` [n_curves][degree+1][dim].

    ``t``: [n_t] (shared) or [n_curves][n_t] (per curve), or None with
    ``t_mode`` UNIFORM / HASH and ``n_t`` given.  Returns points
    [n_curves][n_t][dim] or polyline lengths [n_curves] (FP32), on the same
    device as ``ctrl``.  ``tex_share``: COISSUE only, samples of every 8
    read through the texture unit (1..7, 0 = library default).
    ``tex_format``: texel format of the texture variants (AUTO, UNORM16,
    UNORM8).  ``tex_spread``: TEX_SEILER degree 2, 3 only, texel intervals
    per tile axis of the spread Seiler tile (0 / 1: the paper's 2x2 tile)."""
    n_curves, d1, dim = ctrl.shape
    if t_mode is None:
        t_mode = TMode.SHARED if (t is not None and t.ndim == 1) else TMode.PER_CURVE
    if t is not None:
        n_t = t.shape[-1]
    assert n_t is not None, "n_t is required when t is None"
    shape = (n_curves, n_t, dim) if out_mode == OutMode.POINTS else (n_curves,)
    if out is None:
        out = _empty_like_location(ctrl, shape)
    dev = ctrl.device.index if _is_cuda(ctrl) else (ctx.device if ctx else 0)
    c = ctx or context(dev)
    o = _opts(variant, _dtype_code(ctrl), out_mode, t_mode, seed, stream_id, sync, tex_share, tex_format, tex_spread)
    _check(lib().bez_eval(c.handle, _ptr(ctrl), n_curves, d1 - 1, dim, _ptr(t), n_t, _ptr(out), ctypes.byref(o),
                          _stream_handle(stream, dev)))
    return out


def bez_probe_filter(xyz, *, out=None, stream=None, ctx=None):
    """Sample a 2x2x2 texture whose texel (x, y, z) holds (x, y, z, 1) at the
    unnormalised coordinates ``xyz`` [n][3]; returns the filtered values
    [n][4]: the weight on index 1 along each axis and the weight sum."""
    n = xyz.shape[0]
    if out is None:
        out = _empty_like_location(xyz, (n, 4))
    dev = xyz.device.index if _is_cuda(xyz) else (ctx.device if ctx else 0)
    c = ctx or context(dev)
    _check(lib().bez_probe_filter(c.handle, _ptr(xyz), n, _ptr(out), _stream_handle(stream, dev)))
    return out


def bez_probe_filter_2d(xy, *, out=None, stream=None, ctx=None):
    """Bilinear read of a 2x2 texture with one-hot texels at the unnormalised
    coordinates ``xy`` [n][2]; returns the four texel weights [n][4] (w00,
    w10, w01, w11)."""
    n = xy.shape[0]
    if out is None:
        out = _empty_like_location(xy, (n, 4))
    dev = xy.device.index if _is_cuda(xy) else (ctx.device if ctx else 0)
    c = ctx or context(dev)
    _check(lib().bez_probe_filter_2d(c.handle, _ptr(xy), n, _ptr(out), _stream_handle(stream, dev)))
    return out


def bez_eval_piecewise(ctrl, n_seg, degree, t=None, *, n_t=None, variant=Variant.AUTO, out_mode=OutMode.POINTS,
                       t_mode=None, seed=0, stream_id=0, out=None, stream=None, sync=False, ctx=None,
                       tex_format=TexFormat.AUTO, tex_spread=0):
    """Evaluate C0 chains ``ctrl`` [n_chains][n_seg*degree+1][dim] at global
    parameters in [0, n_seg].  ``tex_spread``: TEX_DECASTELJAU only, texel
    intervals per window axis of the zig-zag texture (0 / 1: (N+1) x 2)."""
    n_chains, n_pts, dim = ctrl.shape
    assert n_pts == n_seg * degree + 1, "ctrl must hold n_seg*degree+1 points per chain"
    if t_mode is None:
        t_mode = TMode.SHARED if (t is not None and t.ndim == 1) else TMode.PER_CURVE
    if t is not None:
        n_t = t.shape[-1]
    assert n_t is not None, "n_t is required when t is None"
    shape = (n_chains, n_t, dim) if out_mode == OutMode.POINTS else (n_chains,)
    if out is None:
        out = _empty_like_location(ctrl, shape)
    dev = ctrl.device.index if _is_cuda(ctrl) else (ctx.device if ctx else 0)
    c = ctx or context(dev)
    o = _opts(variant, _dtype_code(ctrl), out_mode, t_mode, seed, stream_id, sync, 0, tex_format, tex_spread)
    _check(lib().bez_eval_piecewise(c.handle, _ptr(ctrl), n_chains, n_seg, degree, dim, _ptr(t), n_t, _ptr(out),
                                    ctypes.byref(o), _stream_handle(stream, dev)))
    return out


def _spline_call(ctrl, degree, t, n_t, weights, knots, out_mode, t_mode, seed, stream_id, out, stream, sync, ctx,
                 err_word=None):
    n_curves, n_ctrl, dim = ctrl.shape
    if t_mode is None:
        t_mode = TMode.SHARED if (t is not None and t.ndim == 1) else TMode.PER_CURVE
    if t is not None:
        n_t = t.shape[-1]
    assert n_t is not None, "n_t is required when t is None"
    shape = (n_curves, n_t, dim) if out_mode == OutMode.POINTS else (n_curves,)
    if out is None:
        out = _empty_like_location(ctrl, shape)
    dev = ctrl.device.index if _is_cuda(ctrl) else (ctx.device if ctx else 0)
    c = ctx or context(dev)
    o = _opts(Variant.AUTO, _dtype_code(ctrl), out_mode, t_mode, seed, stream_id, sync)
    if err_word is not None:
        o.err_word = _ptr(err_word)
    if weights is None:
        _check(lib().bez_eval_bspline(c.handle, _ptr(ctrl), _ptr(knots), n_curves, n_ctrl, degree, dim, _ptr(t), n_t,
                                      _ptr(out), ctypes.byref(o), _stream_handle(stream, dev)))
    else:
        _check(lib().bez_eval_nurbs(c.handle, _ptr(ctrl), _ptr(weights), _ptr(knots), n_curves, n_ctrl, degree, dim,
                                    _ptr(t), n_t, _ptr(out), ctypes.byref(o), _stream_handle(stream, dev)))
    return out


def bez_eval_bspline(ctrl, degree, t=None, *, knots=None, n_t=None, out_mode=OutMode.POINTS, t_mode=None, seed=0,
                     stream_id=0, out=None, stream=None, sync=False, ctx=None):
    """B-splines ``ctrl`` [n_curves][n_ctrl][dim]; ``knots`` [n_curves][n_ctrl+degree+1] or None
    (clamped uniform)."""
    return _spline_call(ctrl, degree, t, n_t, None, knots, out_mode, t_mode, seed, stream_id, out, stream, sync, ctx)


def bez_eval_nurbs(ctrl, weights, degree, t=None, *, knots=None, n_t=None, out_mode=OutMode.POINTS, t_mode=None,
                   seed=0, stream_id=0, out=None, stream=None, sync=False, ctx=None, err_word=None):
    """NURBS ``ctrl`` [n_curves][n_ctrl][dim] with ``weights`` [n_curves][n_ctrl]."""
    return _spline_call(ctrl, degree, t, n_t, weights, knots, out_mode, t_mode, seed, stream_id, out, stream, sync,
                        ctx, err_word)


def bez_eval_spline_noalloc(ctrl, degree, t=None, *, weights=None, knots=None, n_t=None, out_mode=OutMode.POINTS,
                            t_mode=None, seed=0, stream_id=0, out=None, stream=None, sync=False):
    """B-spline (weights None) or NURBS evaluation through the entry point
    that allocates nothing: every tensor must be on the GPU, and ``out``
    should be preallocated by callers that must not allocate either."""
    n_curves, n_ctrl, dim = ctrl.shape
    if t_mode is None:
        t_mode = TMode.SHARED if (t is not None and t.ndim == 1) else TMode.PER_CURVE
    if t is not None:
        n_t = t.shape[-1]
    assert n_t is not None, "n_t is required when t is None"
    if out is None:
        shape = (n_curves, n_t, dim) if out_mode == OutMode.POINTS else (n_curves,)
        out = _empty_like_location(ctrl, shape)
    dev = _common_device(ctrl, weights, knots, t, out)
    o = _opts(Variant.AUTO, _dtype_code(ctrl), out_mode, t_mode, seed, stream_id, sync)
    if dev is None:
        # host arrays: the library refuses them (it stages nothing)
        _check(lib().bez_eval_spline_noalloc(_ptr(ctrl), _ptr(weights), _ptr(knots), n_curves, n_ctrl, degree,
                                             dim, _ptr(t), n_t, _ptr(out), ctypes.byref(o), None))
        return out
    torch = _torch()
    with torch.cuda.device(dev):
        # the entry point runs on the current device; make it the arrays' one
        _check(lib().bez_eval_spline_noalloc(_ptr(ctrl), _ptr(weights), _ptr(knots), n_curves, n_ctrl, degree,
                                             dim, _ptr(t), n_t, _ptr(out), ctypes.byref(o),
                                             _stream_handle(stream, dev)))
    return out


def _common_device(*arrays):
    """CUDA device index shared by the CUDA tensors among ``arrays`` (None
    entries skipped), or None when none is on a GPU; raises BezError
    (INVALID_ARG) when they sit on different GPUs."""
    devs = {a.device.index for a in arrays if _is_cuda(a)}
    if len(devs) > 1:
        raise BezError(Status.INVALID_ARG, f"arrays on different GPUs: {sorted(devs)}")
    return devs.pop() if devs else None


def bez_eval_surface(ctrl, nu, nv, *, variant=Variant.AUTO, out=None, stream=None, sync=False, ctx=None,
                     tex_format=TexFormat.AUTO, tex_spread=0):
    """Tensor-product surfaces ``ctrl`` [n][du+1][dv+1][dim] on an nu x nv
    uniform grid -> [n][nu][nv][dim].  ``tex_format``: texel storage of the
    texture variants (UNORM16 / UNORM8 with per-tile rescaling)."""
    n, du1, dv1, dim = ctrl.shape
    if out is None:
        out = _empty_like_location(ctrl, (n, nu, nv, dim))
    dev = ctrl.device.index if _is_cuda(ctrl) else (ctx.device if ctx else 0)
    c = ctx or context(dev)
    o = _opts(variant, _dtype_code(ctrl), OutMode.POINTS, TMode.UNIFORM, 0, 0, sync, tex_format=tex_format,
              tex_spread=tex_spread)
    _check(lib().bez_eval_surface(c.handle, _ptr(ctrl), n, du1 - 1, dv1 - 1, dim, nu, nv, _ptr(out),
                                  ctypes.byref(o), _stream_handle(stream, dev)))
    return out


def bez_eval_volume(ctrl, nu, nv, nw, *, variant=Variant.AUTO, out=None, stream=None, sync=False, ctx=None,
                    tex_format=TexFormat.AUTO, tex_spread=0):
    """Tensor-product volumes ``ctrl`` [n][du+1][dv+1][dw+1][dim] on an
    nu x nv x nw uniform grid -> [n][nu][nv][nw][dim].  ``tex_format``: texel
    storage of the texture variants (tricubic scalar volumes)."""
    n, du1, dv1, dw1, dim = ctrl.shape
    if out is None:
        out = _empty_like_location(ctrl, (n, nu, nv, nw, dim))
    dev = ctrl.device.index if _is_cuda(ctrl) else (ctx.device if ctx else 0)
    c = ctx or context(dev)
    o = _opts(variant, _dtype_code(ctrl), OutMode.POINTS, TMode.UNIFORM, 0, 0, sync, tex_format=tex_format,
              tex_spread=tex_spread)
    _check(lib().bez_eval_volume(c.handle, _ptr(ctrl), n, du1 - 1, dv1 - 1, dw1 - 1, dim, nu, nv, nw, _ptr(out),
                                 ctypes.byref(o), _stream_handle(stream, dev)))
    return out


def bez_eval_backward(ctrl, t, grad_out, *, weights=None, need_ctrl=True, need_weights=None, need_t=True,
                      stream=None, sync=False, ctx=None):
    """Adjoint of Bezier (or rational Bezier) evaluation.  Returns
    (grad_ctrl, grad_weights, grad_t); entries not requested are None."""
    n_curves, d1, dim = ctrl.shape
    n_t = t.shape[-1]
    t_mode = TMode.SHARED if t.ndim == 1 else TMode.PER_CURVE
    if need_weights is None:
        need_weights = weights is not None
    gc = _empty_like_location(ctrl, (n_curves, d1, dim)) if need_ctrl else None
    gw = _empty_like_location(ctrl, (n_curves, d1)) if need_weights else None
    gt = _empty_like_location(ctrl, tuple(t.shape)) if need_t else None
    dev = ctrl.device.index if _is_cuda(ctrl) else (ctx.device if ctx else 0)
    c = ctx or context(dev)
    o = _opts(Variant.AUTO, _dtype_code(ctrl), OutMode.POINTS, t_mode, 0, 0, sync)
    _check(lib().bez_eval_backward(c.handle, _ptr(ctrl), _ptr(weights), n_curves, d1 - 1, dim, _ptr(t), n_t,
                                   _ptr(grad_out), _ptr(gc), _ptr(gw), _ptr(gt), ctypes.byref(o),
                                   _stream_handle(stream, dev)))
    return gc, gw, gt


def bez_mse_grad(ctrl, t, target, *, weights=None, loss_scale=None, need_ctrl=True, need_weights=None, need_t=True,
                 stream=None, sync=False, ctx=None):
    """Fused squared-error fit step: per-curve loss s * sum_j ||C(t_j) - target_j||^2
    and its gradients (as bez_eval_backward with grad_out = 2 s (C - target)).
    loss_scale defaults to 1 / target.numel() (mean squared error).  Returns
    (loss [n_curves], grad_ctrl, grad_weights, grad_t); entries not requested
    are None."""
    n_curves, d1, dim = ctrl.shape
    n_t = t.shape[-1]
    t_mode = TMode.SHARED if t.ndim == 1 else TMode.PER_CURVE
    if need_weights is None:
        need_weights = weights is not None
    if loss_scale is None:
        loss_scale = 1.0 / max(1, n_curves * n_t * dim)
    loss = _empty_like_location(ctrl, (n_curves,))
    gc = _empty_like_location(ctrl, (n_curves, d1, dim)) if need_ctrl else None
    gw = _empty_like_location(ctrl, (n_curves, d1)) if need_weights else None
    gt = _empty_like_location(ctrl, tuple(t.shape)) if need_t else None
    dev = ctrl.device.index if _is_cuda(ctrl) else (ctx.device if ctx else 0)
    c = ctx or context(dev)
    L = lib()
    if not getattr(L, "_mse_ready", False):
        L.bez_mse_grad.argtypes = [_VP, _VP, _VP, _I64, _INT, _INT, _VP, _I64, _VP, ctypes.c_float, _VP, _VP, _VP,
                                   _VP, ctypes.POINTER(Opts), _VP]
        L.bez_mse_grad.restype = ctypes.c_int
        L._mse_ready = True
    o = _opts(Variant.AUTO, _dtype_code(ctrl), OutMode.POINTS, t_mode, 0, 0, sync)
    _check(L.bez_mse_grad(c.handle, _ptr(ctrl), _ptr(weights), n_curves, d1 - 1, dim, _ptr(t), n_t, _ptr(target),
                          float(loss_scale), _ptr(loss), _ptr(gc), _ptr(gw), _ptr(gt), ctypes.byref(o),
                          _stream_handle(stream, dev)))
    return loss, gc, gw, gt


# ---------------------------------------------------------------- mixed batches

DESC_DTYPE = np.dtype([("type", "<i4"), ("degree", "<i4"), ("n_ctrl", "<i4"), ("n_samples", "<i4"),
                       ("ctrl_off", "<i8"), ("weight_off", "<i8"), ("out_off", "<i8")])


class BatchOpts(ctypes.Structure):
    _fields_ = [("autotune", ctypes.c_int32), ("setup_each_launch", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("schedule", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("repr", ctypes.c_int32)]


def descriptors(type, degree, n_ctrl, n_samples, ctrl_off, weight_off, out_off):
    """Pack per-curve arrays into the C descriptor layout (NumPy, host)."""
    d = np.zeros(len(type), DESC_DTYPE)
    d["type"], d["degree"], d["n_ctrl"], d["n_samples"] = type, degree, n_ctrl, n_samples
    d["ctrl_off"], d["weight_off"], d["out_off"] = ctrl_off, weight_off, out_off
    return d


def _batch_lib():
    L = lib()
    if not getattr(L, "_batch_ready", False):
        L.bez_batch_create.argtypes = [_VP, _VP, _I64, _INT, _VP, _I64, _VP, _I64, _VP, _I64,
                                       ctypes.POINTER(BatchOpts), _VP, ctypes.POINTER(_VP)]
        L.bez_batch_launch.argtypes = [_VP, _VP]
        L.bez_batch_config.argtypes = [_VP] + [ctypes.POINTER(ctypes.c_int32)] * 4
        L.bez_batch_destroy.argtypes = [_VP]
        L.bez_eval_batch.argtypes = [_VP, _VP, _I64, _INT, _VP, _I64, _VP, _I64, _VP, _I64, _VP]
        for n in ("bez_batch_create", "bez_batch_launch", "bez_batch_config", "bez_batch_destroy", "bez_eval_batch"):
            getattr(L, n).restype = ctypes.c_int
        L._batch_ready = True
    return L


def _numel(x):
    return 0 if x is None else int(x.numel() if not isinstance(x, np.ndarray) else x.size)


class Batch:
    """A mixed-batch plan (bez_batch_create); ``launch()`` replays it."""

    def __init__(self, desc, dim, ctrl_pool, weight_pool, out_pool, *, autotune=False, setup_each_launch=True,
                 use_graph=True, chunk=0, schedule=-1, threads=0, repr=-1, stream=None, ctx=None):
        L = _batch_lib()
        desc = np.ascontiguousarray(desc, dtype=DESC_DTYPE)
        self.dev = ctrl_pool.device.index
        self.ctx = ctx or context(self.dev)
        self._keep = (ctrl_pool, weight_pool, out_pool)
        bo = BatchOpts(int(autotune), int(setup_each_launch), int(use_graph), chunk, schedule, threads, repr)
        h = _VP()
        _check(L.bez_batch_create(self.ctx.handle, desc.ctypes.data, len(desc), dim, _ptr(ctrl_pool),
                                  _numel(ctrl_pool), _ptr(weight_pool), _numel(weight_pool), _ptr(out_pool),
                                  _numel(out_pool), ctypes.byref(bo), _stream_handle(stream, self.dev),
                                  ctypes.byref(h)))
        self.handle = h

    def launch(self, stream=None):
        _check(_batch_lib().bez_batch_launch(self.handle, _stream_handle(stream, self.dev)))

    def config(self):
        c, s, t, r = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(_batch_lib().bez_batch_config(self.handle, ctypes.byref(c), ctypes.byref(s), ctypes.byref(t),
                                             ctypes.byref(r)))
        return {"chunk": c.value, "schedule": s.value, "threads": t.value, "repr": r.value}

    def close(self):
        if getattr(self, "handle", None):
            _batch_lib().bez_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bez_eval_batch(desc, dim, ctrl_pool, weight_pool, out_pool, *, stream=None, ctx=None):
    """One-shot mixed batch (no graph, no tuning), synchronous on the stream."""
    L = _batch_lib()
    desc = np.ascontiguousarray(desc, dtype=DESC_DTYPE)
    dev = ctrl_pool.device.index
    c = ctx or context(dev)
    _check(L.bez_eval_batch(c.handle, desc.ctypes.data, len(desc), dim, _ptr(ctrl_pool), _numel(ctrl_pool),
                            _ptr(weight_pool), _numel(weight_pool), _ptr(out_pool), _numel(out_pool),
                            _stream_handle(stream, dev)))
    return out_pool


PEAK_KINDS = {"fma": 0, "tex2d_f32": 1, "tex2d_f16": 2, "tex3d_f32": 3, "tex3d_f16": 4, "store": 5, "copy": 6}


def bez_measure_peak(kind, *, stream=None, ctx=None):
    """Run one peak microbenchmark (see include/bez.h): FMA lane-ops/s,
    texture fetches/s, or memory GB/s."""
    L = lib()
    if not getattr(L, "_peak_ready", False):
        L.bez_measure_peak.argtypes = [_VP, _INT, ctypes.POINTER(ctypes.c_double), _VP]
        L.bez_measure_peak.restype = ctypes.c_int
        L._peak_ready = True
    c = ctx or context()
    v = ctypes.c_double()
    _check(L.bez_measure_peak(c.handle, PEAK_KINDS[kind], ctypes.byref(v), _stream_handle(stream, c.device)))
    return v.value
