"""Pins for the oracle's B-spline / NURBS, surface / volume and gradient
functions (CPU only).

B-splines: Boehm knot insertion to Bezier spans + exact de Casteljau (the
paper's Sec. 2.2 route, in rational arithmetic), SciPy's BSpline, the closed
form of the uniform cubic basis, and the reduction n = p + 1 -> Bezier.
NURBS: quarter circle, unit weights -> B-spline, weight scaling invariance.
Surfaces / volumes: einsum with Bernstein matrices taken from SciPy's
binomial pmf (B_i^d(t) = binom.pmf(i, d, t)), and reduction to a curve.
Gradients: linearity (grad_ctrl = B^T g), central finite differences in FP64
and torch's CPU autograd through an independent Bernstein sum."""
import json
import os
import random
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
from exact import bspline_via_boehm, clamped_uniform_knots_exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_clamped_uniform_knots():
    for n, p in [(4, 3), (7, 3), (10, 2), (64, 3), (9, 7)]:
        U = oracle.clamped_uniform_knots(n, p)
        np.testing.assert_array_equal(U, np.array([float(x) for x in clamped_uniform_knots_exact(n, p)]))


@pytest.mark.parametrize("n,p", [(4, 3), (6, 3), (9, 3), (7, 2), (8, 5)])
def test_bspline_equals_boehm_extraction(n, p):
    rng = random.Random(100 * n + p)
    U = clamped_uniform_knots_exact(n, p)
    P = [F(rng.randint(-8, 8)) for _ in range(n)]
    us = [F(k, 4 * (n - p) * 3) for k in range(0, 4 * (n - p) * 3 + 1)]
    got = oracle.bspline(np.array([[[float(v)] for v in P]]), p, np.array([float(u) for u in us]))
    for j, u in enumerate(us):
        assert got[0, j, 0] == pytest.approx(float(bspline_via_boehm(U, P, p, u)), abs=1e-13)


def test_bspline_scipy_and_general_knots():
    from scipy.interpolate import BSpline
    rng = np.random.default_rng(21)
    for p in (1, 2, 3, 4):
        n = 11
        inner = np.sort(rng.uniform(0, 1, n - p - 1))
        U = np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])
        ctrl = rng.uniform(-1, 1, size=(1, n, 3))
        t = np.concatenate([rng.uniform(0, 1, 200), [0.0, 1.0]])
        got = oracle.bspline(ctrl, p, t, knots=U[None])
        want = BSpline(U, ctrl[0], p)(t)
        np.testing.assert_allclose(got[0], want, rtol=0, atol=1e-13)


def test_bspline_uniform_cubic_basis_golden():
    gold = json.load(open(os.path.join(GOLDEN, "uniform_cubic_bspline.json")))
    U = np.arange(8, dtype=np.float64)[None]          # uniform knots, one span [3, 4]
    ctrl = np.eye(4)[None]                             # P_i = e_i exposes the basis
    ts = [a / b for a, b in gold["t"]]
    got = oracle.bspline(ctrl, 3, np.array([3.0 + t for t in ts]), knots=U)
    want = np.array([[a / b for a, b in row] for row in gold["basis"]])
    np.testing.assert_allclose(got[0], want, rtol=0, atol=1e-15)


def test_bspline_single_span_is_bezier_and_partition():
    rng = np.random.default_rng(22)
    for p in range(1, 8):
        ctrl = rng.uniform(-1, 1, size=(3, p + 1, 3))
        t = rng.uniform(0, 1, 100)
        np.testing.assert_allclose(oracle.bspline(ctrl, p, t), oracle.bezier(ctrl, t), rtol=0, atol=1e-14)
    c = np.full((1, 20, 3), 0.37)
    np.testing.assert_allclose(oracle.bspline(c, 3, rng.uniform(0, 1, 50)), 0.37, rtol=0, atol=1e-15)
    ctrl = rng.uniform(-1, 1, size=(2, 12, 3))
    out = oracle.bspline(ctrl, 3, np.array([0.0, 1.0, -1.0, 2.0]))
    np.testing.assert_array_equal(out[:, 0], ctrl[:, 0])
    np.testing.assert_array_equal(out[:, 1], ctrl[:, -1])
    np.testing.assert_array_equal(out[:, 2], ctrl[:, 0])
    np.testing.assert_array_equal(out[:, 3], ctrl[:, -1])


def test_nurbs_quarter_circle_and_reductions():
    gold = json.load(open(os.path.join(GOLDEN, "quarter_circle_nurbs.json")))
    ctrl = np.array([gold["ctrl"]], np.float64)
    w = np.array([gold["weights"]])
    t = np.linspace(0, 1, 33)
    pts = oracle.bspline(ctrl, 2, t, weights=w)
    np.testing.assert_allclose(np.linalg.norm(pts[0], axis=1), 1.0, atol=1e-15)
    rng = np.random.default_rng(23)
    c = rng.uniform(-1, 1, size=(3, 15, 3))
    t = rng.uniform(0, 1, 80)
    np.testing.assert_allclose(oracle.bspline(c, 3, t, weights=np.ones((3, 15))), oracle.bspline(c, 3, t),
                               atol=1e-15)
    w = rng.uniform(0.5, 2, (3, 15))
    np.testing.assert_allclose(oracle.bspline(c, 3, t, weights=4 * w), oracle.bspline(c, 3, t, weights=w),
                               atol=1e-14)
    # homogeneous form: NURBS = (B-spline of w P) / (B-spline of w)
    num = oracle.bspline(c * w[:, :, None], 3, t)
    den = oracle.bspline(w[:, :, None], 3, t)
    np.testing.assert_allclose(oracle.bspline(c, 3, t, weights=w), num / den, atol=1e-14)


# ------------------------------------------------------------------ tensor products

def _bernstein_matrix(d, t):
    from scipy.stats import binom
    return np.stack([binom.pmf(i, d, t) for i in range(d + 1)], axis=1)  # [len(t)][d+1]


def test_surface_against_scipy_basis_einsum():
    rng = np.random.default_rng(31)
    for du, dv in [(3, 3), (1, 2), (4, 2)]:
        ctrl = rng.uniform(-1, 1, size=(3, du + 1, dv + 1, 3))
        nu, nv = 9, 7
        Bu = _bernstein_matrix(du, oracle.grid(nu))
        Bv = _bernstein_matrix(dv, oracle.grid(nv))
        want = np.einsum("ui,nijk,vj->nuvk", Bu, ctrl, Bv)
        np.testing.assert_allclose(oracle.surface(ctrl, nu, nv), want, rtol=0, atol=1e-14)


def test_surface_edges_reduce_to_curves():
    rng = np.random.default_rng(32)
    ctrl = rng.uniform(-1, 1, size=(2, 4, 4, 3))
    S = oracle.surface(ctrl, 5, 6)
    np.testing.assert_allclose(S[:, :, 0], oracle.bezier_grid(ctrl[:, :, 0], 5), atol=1e-15)   # v = 0
    np.testing.assert_allclose(S[:, 0, :], oracle.bezier_grid(ctrl[:, 0, :], 6), atol=1e-15)   # u = 0
    np.testing.assert_array_equal(S[:, 0, 0], ctrl[:, 0, 0])
    np.testing.assert_array_equal(S[:, -1, -1], ctrl[:, -1, -1])


def test_volume_against_scipy_basis_einsum():
    rng = np.random.default_rng(33)
    ctrl = rng.normal(size=(3, 4, 4, 4, 1))
    n = 5
    B = _bernstein_matrix(3, oracle.grid(n))
    want = np.einsum("ai,bj,cl,nijlk->nabck", B, B, B, ctrl)
    np.testing.assert_allclose(oracle.volume(ctrl, n, n, n), want, rtol=0, atol=1e-14)
    ctrl2 = rng.normal(size=(2, 2, 3, 4, 2))
    B1, B2, B3 = (_bernstein_matrix(d, oracle.grid(m)) for d, m in [(1, 3), (2, 4), (3, 5)])
    want2 = np.einsum("ai,bj,cl,nijlk->nabck", B1, B2, B3, ctrl2)
    np.testing.assert_allclose(oracle.volume(ctrl2, 3, 4, 5), want2, rtol=0, atol=1e-14)


# ------------------------------------------------------------------ gradients

def test_grad_ctrl_is_basis_transpose_times_g():
    rng = np.random.default_rng(41)
    d, B, n_t = 3, 4, 37
    ctrl = rng.uniform(-1, 1, (B, d + 1, 3))
    t = rng.uniform(0, 1, (B, n_t))
    g = rng.normal(size=(B, n_t, 3))
    gc, gw, gt = oracle.bezier_grad(ctrl, t, g)
    assert gw is None
    for c in range(B):
        Bm = _bernstein_matrix(d, t[c])                   # [n_t][d+1]
        np.testing.assert_allclose(gc[c], Bm.T @ g[c], rtol=0, atol=1e-13)


@pytest.mark.parametrize("rational", [False, True])
def test_grad_finite_differences(rational):
    rng = np.random.default_rng(42 + rational)
    d, B, n_t = 4, 2, 9
    ctrl = rng.uniform(-1, 1, (B, d + 1, 3))
    w = rng.uniform(0.5, 2, (B, d + 1)) if rational else None
    t = rng.uniform(0.05, 0.95, (B, n_t))
    g = rng.normal(size=(B, n_t, 3))
    gc, gw, gt = oracle.bezier_grad(ctrl, t, g, weights=w)
    h = 1e-6

    def loss(c_, w_, t_):
        return float(np.sum(oracle.bezier(c_, t_, weights=w_) * g))

    for c in range(B):
        for i in range(d + 1):
            for k in range(3):
                e = np.zeros_like(ctrl)
                e[c, i, k] = h
                fd = (loss(ctrl + e, w, t) - loss(ctrl - e, w, t)) / (2 * h)
                assert gc[c, i, k] == pytest.approx(fd, abs=1e-8)
            if rational:
                e = np.zeros_like(w)
                e[c, i] = h
                fd = (loss(ctrl, w + e, t) - loss(ctrl, w - e, t)) / (2 * h)
                assert gw[c, i] == pytest.approx(fd, abs=1e-8)
        for j in range(n_t):
            e = np.zeros_like(t)
            e[c, j] = h
            fd = (loss(ctrl, w, t + e) - loss(ctrl, w, t - e)) / (2 * h)
            assert gt[c, j] == pytest.approx(fd, abs=1e-8)


def test_grad_against_torch_autograd_and_shared_t():
    torch = pytest.importorskip("torch")
    from math import comb
    rng = np.random.default_rng(43)
    d, B, n_t = 5, 3, 11
    ctrl = rng.uniform(-1, 1, (B, d + 1, 3))
    w = rng.uniform(0.5, 2, (B, d + 1))
    t = rng.uniform(0, 1, n_t)
    g = rng.normal(size=(B, n_t, 3))
    tc = torch.tensor(ctrl, requires_grad=True)
    tw = torch.tensor(w, requires_grad=True)
    tt = torch.tensor(t, requires_grad=True)
    basis = torch.stack([comb(d, i) * (1 - tt) ** (d - i) * tt ** i for i in range(d + 1)], dim=1)  # [n_t][d+1]
    num = torch.einsum("ji,ci,cik->cjk", basis, tw, tc)
    den = torch.einsum("ji,ci->cj", basis, tw)
    pts = num / den[:, :, None]
    (pts * torch.tensor(g)).sum().backward()
    gc, gw, gt = oracle.bezier_grad(ctrl, t, g, weights=w)
    np.testing.assert_allclose(gc, tc.grad.numpy(), atol=1e-13)
    np.testing.assert_allclose(gw, tw.grad.numpy(), atol=1e-13)
    np.testing.assert_allclose(gt, tt.grad.numpy(), atol=1e-12)   # shared t: summed over curves


def test_grad_t_zero_where_clamped():
    ctrl = np.random.default_rng(44).uniform(-1, 1, (1, 4, 3))
    g = np.ones((1, 3, 3))
    _, _, gt = oracle.bezier_grad(ctrl, np.array([[-0.25, 0.5, 1.25]]), g)
    assert gt[0, 0] == 0.0 and gt[0, 2] == 0.0 and gt[0, 1] != 0.0
