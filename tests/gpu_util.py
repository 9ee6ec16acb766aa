"""Helpers for the GPU parity tests: device checks, the normalised error of
the accuracy bar, and a-priori FP32 error bounds derived from the arithmetic.

Normalised error (per curve): max_j |P_gpu - P_ref|_2 / max(diag, 2^-4), with
diag the bounding-box diagonal of the FP64 oracle points of that curve; the
floor keeps nearly-degenerate curves from turning FP32 coordinate rounding
into a large relative figure.
"""
from math import comb

import numpy as np
import pytest

U32 = 2.0 ** -24
DELTA = 2.0 ** -4


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_15447_gb300 import build
    build.build()
    return torch


def curve_diag(ref):
    """ref [B][n][dim] -> [B] bounding-box diagonal of the oracle points."""
    lo = ref.min(axis=1)
    hi = ref.max(axis=1)
    return np.linalg.norm(hi - lo, axis=-1)


def normalised_error(got, ref):
    """Per-curve max point error over max(diag, 2^-4)."""
    got = np.asarray(got, np.float64)
    err = np.linalg.norm(got - ref, axis=-1)          # [B][n]
    with np.errstate(invalid="ignore"):
        return err.max(axis=1) / np.maximum(curve_diag(ref), DELTA)


def gamma(n):
    return n * U32 / (1 - n * U32)


def horner_bound(ctrl, t):
    """A-priori bound on |Horner_fp32(t) - C(t)| per point and component for
    the power basis about 0 built by forward differences: rounding of the
    coefficients a_k = binom(d,k) Delta^k b_0 (gamma_(k+1) 2^k max|b| binom)
    plus Horner's own gamma_(2d) sum |a_k| t^k.  ctrl [B][d+1][dim] FP64,
    t [n] or [B][n].  Returns [B][n][dim]."""
    B, d1, dim = ctrl.shape
    d = d1 - 1
    diffs = ctrl.copy()
    a = np.empty_like(ctrl)
    for k in range(d + 1):
        a[:, k] = comb(d, k) * diffs[:, 0]
        diffs = diffs[:, 1:] - diffs[:, :-1]
    M = np.abs(ctrl).max(axis=1)                      # [B][dim]
    tt = np.broadcast_to(np.abs(t), (B, np.shape(t)[-1]))
    powk = np.stack([tt ** k for k in range(d + 1)], axis=-1)   # [B][n][d+1]
    horner = gamma(2 * d + 1) * np.einsum("bnk,bkc->bnc", powk, np.abs(a))
    conv_k = np.array([comb(d, k) * (gamma(k + 1) * 2 ** k + U32) for k in range(d + 1)])
    conv = np.einsum("bnk,k,bc->bnc", powk, conv_k, M) * 2
    return horner + conv + 1e-30


def normalised_error_ctrl(got, ref, ctrl):
    """Secondary normaliser: per-curve max point error over the diagonal of
    the control polygon's bounding box (floor 2^-4).  Used for point
    dimensions other than 3, where a curve's sampled range can be far
    smaller than its control values (a scalar polynomial with a flat stretch)
    and the primary normaliser becomes ill-conditioned."""
    got = np.asarray(got, np.float64)
    err = np.linalg.norm(got - ref, axis=-1)
    c = np.asarray(ctrl, np.float64)
    diag = np.linalg.norm(c.max(axis=1) - c.min(axis=1), axis=-1)
    return err.max(axis=1) / np.maximum(diag, DELTA)
