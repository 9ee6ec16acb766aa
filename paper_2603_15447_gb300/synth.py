"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
runs.  This module only draws numbers: it holds none of the evaluation
arithmetic, and neither the CUDA path nor the oracle depends on it.

Every value is a pure function of (seed, stream, index) through Wellons'
lowbias32 mixer, so CPU and GPU consumers see bit-identical FP32 inputs:

    key      = H(lo(seed) ^ H(hi(seed) ^ H(stream)))
    h_i      = H(key ^ H(i))                      (i < 2^32)
    u_i      = (h_i >> 8) * 2^-24                 (FP32-exact uniform in [0,1))

Uniform [-1,1) values are 2 u - 1 (exact).  Normal values use Box-Muller on
two streams in FP64, rounded once to FP32.

Workload recipes (base seed 20260315 plus the workload index):
  plain       4096 cubic 3D curves U[-1,1]^3, 256 shared t = fl32(j)/fl32(255)
  precision   1,048,576 cubic 3D curves U[-1,1]^3, 1024 t per curve drawn in
              the kernel (lowbias32 of seed, stream, curve, j), fused polyline
              length; chains: 16,384 chains x 64 quadratic segments, t U[0,64)
  batch       262,144 curves: 50% Bezier (degree U{1..7}), 25% clamped uniform
              cubic B-splines (n U{4..64}), 25% NURBS (degree U{1..7},
              n U{max(4,p+1)..64}, w U[0.5,2]); samples floor(exp(U[ln16, ln4096]))
  tensor      65,536 bicubic patches U[-1,1]^3 on 32x32; 4096 tricubic scalar
              volumes N(0,1) on 16^3
  fit         65,536 cubic 3D curves, 512 sorted t U[0,1), targets = truth +
              N(0, 0.01^2) noise; initial control points from another stream
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20260315
M32 = np.uint64(0xFFFFFFFF)


def lowbias32(x):
    x = np.asarray(x, dtype=np.uint32).astype(np.uint64)
    x ^= x >> np.uint64(16)
    x = (x * np.uint64(0x7FEB352D)) & M32
    x ^= x >> np.uint64(15)
    x = (x * np.uint64(0x846CA68B)) & M32
    x ^= x >> np.uint64(16)
    return x.astype(np.uint32)


def key(seed: int, stream: int) -> np.uint32:
    lo = np.uint32(seed & 0xFFFFFFFF)
    hi = np.uint32((seed >> 32) & 0xFFFFFFFF)
    return lowbias32(lo ^ lowbias32(hi ^ lowbias32(np.uint32(stream))))


def bits(seed: int, stream: int, n: int, offset: int = 0):
    k = key(seed, stream)
    idx = np.arange(offset, offset + n, dtype=np.uint64).astype(np.uint32)
    return lowbias32(k ^ lowbias32(idx))


def uniform01(seed, stream, shape):
    n = int(np.prod(shape))
    u = (bits(seed, stream, n) >> np.uint32(8)).astype(np.float32) * np.float32(2.0 ** -24)
    return u.reshape(shape)


def uniform(seed, stream, shape, lo=-1.0, hi=1.0):
    u = uniform01(seed, stream, shape)
    if (lo, hi) == (-1.0, 1.0):
        return (np.float32(2.0) * u - np.float32(1.0)).astype(np.float32)
    return (np.float64(lo) + (np.float64(hi) - np.float64(lo)) * u.astype(np.float64)).astype(np.float32)


def normal(seed, stream, shape):
    n = int(np.prod(shape))
    u1 = uniform01(seed, stream, (n,)).astype(np.float64)
    u2 = uniform01(seed, stream + 0x5BD1E995, (n,)).astype(np.float64)
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    return z.astype(np.float32).reshape(shape)


def randint(seed, stream, n, lo, hi):
    """Integers uniform in [lo, hi] (inclusive)."""
    u = uniform01(seed, stream, (n,)).astype(np.float64)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64).clip(lo, hi)


# ---------------------------------------------------------------- workloads

def plain(seed=BASE_SEED + 0, n_curves=4096, n_t=256, degree=3, dim=3):
    ctrl = uniform(seed, 1, (n_curves, degree + 1, dim))
    t = (np.arange(n_t, dtype=np.float32) / np.float32(max(n_t - 1, 1))).astype(np.float32)
    return ctrl, t


def precision(seed=BASE_SEED + 1, n_curves=1 << 20, degree=3, dim=3):
    """Control points of the fused evaluate-and-measure workload; the
    parameters (1024 per curve) are drawn in the kernel with (seed, stream 2)."""
    return uniform(seed, 1, (n_curves, degree + 1, dim))


PRECISION_T_STREAM = 2
PRECISION_N_T = 1024


def chains(seed=BASE_SEED + 1, n_chains=16384, n_seg=64, n_t=65536, degree=2, dim=3):
    ctrl = uniform(seed, 11, (n_chains, n_seg * degree + 1, dim))
    t = (uniform01(seed, 12, (n_chains, n_t)).astype(np.float64) * n_seg).astype(np.float32)
    t = np.minimum(t, np.float32(n_seg))
    return ctrl, t


def batch(seed=BASE_SEED + 2, n_curves=262144, dim=3, max_samples=4096, min_samples=16):
    """Descriptors of the mixed workload as NumPy arrays:
    type (0 Bezier, 1 B-spline, 2 NURBS), degree, n_ctrl, n_samples, plus the
    control-point and weight pools and offsets."""
    kinds = np.zeros(n_curves, np.int32)
    u = uniform01(seed, 21, (n_curves,))
    kinds[u >= 0.5] = 1
    kinds[u >= 0.75] = 2
    deg = randint(seed, 22, n_curves, 1, 7).astype(np.int32)
    deg[kinds == 1] = 3
    n_bspl = randint(seed, 23, n_curves, 4, 64)
    u_n = uniform01(seed, 24, (n_curves,)).astype(np.float64)
    lo_nurbs = np.maximum(4, deg + 1)
    n_nurbs = (lo_nurbs + np.floor(u_n * (64 - lo_nurbs + 1))).astype(np.int64).clip(lo_nurbs, 64)
    n_ctrl = np.where(kinds == 0, deg + 1, np.where(kinds == 1, n_bspl, n_nurbs)).astype(np.int32)
    us = uniform01(seed, 25, (n_curves,)).astype(np.float64)
    n_samples = np.floor(np.exp(np.log(min_samples) + us * (np.log(max_samples) - np.log(min_samples))))
    n_samples = n_samples.astype(np.int64).clip(min_samples, max_samples).astype(np.int32)
    ctrl_off = np.zeros(n_curves + 1, np.int64)
    ctrl_off[1:] = np.cumsum(n_ctrl.astype(np.int64) * dim)
    w_off = np.zeros(n_curves + 1, np.int64)
    w_off[1:] = np.cumsum(np.where(kinds == 2, n_ctrl, 0).astype(np.int64))
    out_off = np.zeros(n_curves + 1, np.int64)
    out_off[1:] = np.cumsum(n_samples.astype(np.int64) * dim)
    ctrl_pool = uniform(seed, 26, (int(ctrl_off[-1]),))
    weight_pool = uniform(seed, 27, (max(int(w_off[-1]), 1),), 0.5, 2.0)
    return dict(type=kinds, degree=deg, n_ctrl=n_ctrl, n_samples=n_samples, ctrl_off=ctrl_off[:-1],
                weight_off=w_off[:-1], out_off=out_off[:-1], ctrl_pool=ctrl_pool, weight_pool=weight_pool,
                out_len=int(out_off[-1]), dim=dim)


def surfaces(seed=BASE_SEED + 3, n=65536, du=3, dv=3, dim=3):
    return uniform(seed, 31, (n, du + 1, dv + 1, dim))


def volumes(seed=BASE_SEED + 3, n=4096, d=3, dim=1):
    return normal(seed, 32, (n, d + 1, d + 1, d + 1, dim))


def fit(seed=BASE_SEED + 4, n_curves=65536, n_t=512, degree=3, dim=3, sigma=0.01):
    """(truth ctrl, sorted t, noise [n][n_t][dim], init ctrl).  Targets are
    truth(t) + noise, evaluated by whichever evaluator the caller trusts."""
    truth = uniform(seed, 41, (n_curves, degree + 1, dim))
    t = np.sort(uniform01(seed, 42, (n_curves, n_t)), axis=1).astype(np.float32)
    noise = (np.float32(sigma) * normal(seed, 43, (n_curves, n_t, dim))).astype(np.float32)
    init = uniform(seed, 44, (n_curves, degree + 1, dim))
    return truth, t, noise, init
