"""GPU parity of B-spline and NURBS evaluation (bez_eval_bspline /
bez_eval_nurbs, paper Sec. 2.2) against the oracle's Cox-de Boor recursion,
at the FP32 bar (1e-6 of the curve's bounding-box diagonal)."""
import json
import os

import numpy as np
import pytest

import oracle
from gpu_util import need_gpu, normalised_error, normalised_error_ctrl

pytestmark = pytest.mark.gpu
FP32_BAR = 1e-6
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _t(torch, x):
    return None if x is None else torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()


def _bspline(torch, ctrl, p, t=None, knots=None, weights=None, **kw):
    from paper_2603_15447_gb300 import bez
    c = _t(torch, ctrl)
    if weights is None:
        out = bez.bez_eval_bspline(c, p, _t(torch, t), knots=_t(torch, knots), **kw)
    else:
        out = bez.bez_eval_nurbs(c, _t(torch, weights), p, _t(torch, t), knots=_t(torch, knots), **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _random_knots(rng, B, n, p):
    """Clamped knot vectors with random interior knots on a 1/16 grid,
    interior multiplicity at most p."""
    U = np.empty((B, n + p + 1), np.float32)
    for b in range(B):
        while True:
            inner = np.sort(rng.integers(1, 16, n - p - 1)) / 16.0
            vals, counts = np.unique(inner, return_counts=True)
            if counts.size == 0 or counts.max() <= p:
                break
        U[b] = np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])
    return U


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("rational", [False, True])
def test_clamped_uniform(p, rational):
    torch = need_gpu()
    rng = np.random.default_rng(100 * p + rational)
    for n in (p + 1, p + 5, 40):
        ctrl = rng.uniform(-1, 1, size=(301, n, 3)).astype(np.float32)
        w = rng.uniform(0.5, 2, size=(301, n)).astype(np.float32) if rational else None
        t = rng.uniform(0, 1, 67).astype(np.float32)
        t[:4] = [0.0, 1.0, 0.5, 1.0 / (n - p) if n > p + 1 else 0.25]
        got = _bspline(torch, ctrl, p, t, weights=w)
        ref = oracle.bspline(ctrl, p, t, weights=w)
        assert normalised_error(got, ref).max() <= FP32_BAR, n
        np.testing.assert_allclose(got[:, 0], ctrl[:, 0], rtol=0, atol=4e-7)
        np.testing.assert_allclose(got[:, 1], ctrl[:, -1], rtol=0, atol=4e-7)


@pytest.mark.parametrize("p", [1, 2, 3, 5])
@pytest.mark.parametrize("rational", [False, True])
def test_general_knots_per_curve_t(p, rational):
    torch = need_gpu()
    rng = np.random.default_rng(200 + 10 * p + rational)
    n, B = 12, 157
    ctrl = rng.uniform(-1, 1, size=(B, n, 3)).astype(np.float32)
    w = rng.uniform(0.5, 2, size=(B, n)).astype(np.float32) if rational else None
    U = _random_knots(rng, B, n, p)
    t = rng.uniform(0, 1, (B, 53)).astype(np.float32)
    t[:, 0] = U[:, p + 1]                                  # on an interior knot
    got = _bspline(torch, ctrl, p, t, knots=U, weights=w)
    ref = oracle.bspline(ctrl, p, t, weights=w, knots=U)
    assert normalised_error(got, ref).max() <= FP32_BAR


@pytest.mark.parametrize("dim", [1, 2, 4])
def test_other_dims(dim):
    torch = need_gpu()
    rng = np.random.default_rng(300 + dim)
    ctrl = rng.uniform(-1, 1, size=(99, 9, dim)).astype(np.float32)
    w = rng.uniform(0.5, 2, size=(99, 9)).astype(np.float32)
    t = rng.uniform(0, 1, 31).astype(np.float32)
    for weights in (None, w):
        got = _bspline(torch, ctrl, 3, t, weights=weights)
        ref = oracle.bspline(ctrl, 3, t, weights=weights)
        assert normalised_error_ctrl(got, ref, ctrl).max() <= FP32_BAR


def test_uniform_hash_length_modes():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(400)
    ctrl = rng.uniform(-1, 1, size=(120, 20, 3)).astype(np.float32)
    w = rng.uniform(0.5, 2, size=(120, 20)).astype(np.float32)
    got = _bspline(torch, ctrl, 3, n_t=200, weights=w, t_mode=bez.TMode.UNIFORM)
    assert normalised_error(got, oracle.bspline(ctrl, 3, oracle.grid(200), weights=w)).max() <= FP32_BAR
    got = _bspline(torch, ctrl, 3, n_t=64, t_mode=bez.TMode.HASH, seed=8, stream_id=3)
    th = oracle.hash_t(8, 3, 0, 120, 64)
    assert normalised_error(got, oracle.bspline(ctrl, 3, th)).max() <= FP32_BAR
    # general knots: the [0,1) draws map onto [U_p, U_n]
    U = _random_knots(rng, 120, 20, 3)
    U = (U * 2 - 0.5).astype(np.float32)                   # domain [-0.5, 1.5]
    got = _bspline(torch, ctrl, 3, n_t=64, knots=U, t_mode=bez.TMode.HASH, seed=8, stream_id=3)
    tk = (np.float32(2.0) * th.astype(np.float32) + np.float32(-0.5)).astype(np.float32)
    assert normalised_error(got, oracle.bspline(ctrl, 3, tk, knots=U)).max() <= FP32_BAR
    L = _bspline(torch, ctrl, 3, n_t=512, weights=w, t_mode=bez.TMode.UNIFORM,
                 out_mode=bez.OutMode.POLYLINE_LENGTH)
    pts = oracle.bspline(ctrl, 3, oracle.grid(512), weights=w)
    Lref = oracle.polyline_length(pts)
    diag = np.linalg.norm(pts.max(axis=1) - pts.min(axis=1), axis=-1)
    assert np.all(np.abs(L - Lref) <= 2 * 511 * FP32_BAR * diag + 40 * 2.0 ** -24 * Lref)


def test_quarter_circle_and_edge_cases():
    torch = need_gpu()
    gold = json.load(open(os.path.join(GOLDEN, "quarter_circle_nurbs.json")))
    ctrl = np.array([gold["ctrl"]], np.float32)
    w = np.array([gold["weights"]], np.float32)
    t = np.linspace(0, 1, 1001).astype(np.float32)
    got = _bspline(torch, ctrl, 2, t, weights=w)
    r = np.linalg.norm(got[0].astype(np.float64), axis=1)
    # the FP32 weight sqrt(2)/2 moves the exact circle by ~1e-8
    assert np.abs(r - 1).max() <= 1e-6
    rng = np.random.default_rng(500)
    ctrl = rng.uniform(-1, 1, size=(10, 8, 3)).astype(np.float32)
    got = _bspline(torch, ctrl, 3, np.array([-1.0, 2.0, np.nan], np.float32))
    ref = oracle.bspline(ctrl, 3, np.array([0.0, 1.0]))
    np.testing.assert_allclose(got[:, :2], ref, rtol=0, atol=4e-7)
    assert np.isnan(got[:, 2]).all()


def test_zero_weights_counted():
    torch = need_gpu()
    rng = np.random.default_rng(600)
    ctrl = rng.uniform(-1, 1, size=(4, 6, 3)).astype(np.float32)
    w = np.zeros((4, 6), np.float32)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    from paper_2603_15447_gb300 import bez
    bez.bez_eval_nurbs(_t(torch, ctrl), _t(torch, w), 3, _t(torch, np.linspace(0, 1, 10)), err_word=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 40


def test_spline_argument_errors():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval_bspline(torch.zeros((2, 3, 3), device="cuda"), 3, torch.zeros(4, device="cuda"))
    assert e.value.status == bez.Status.INVALID_ARG
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval_bspline(torch.zeros((2, 8, 3), device="cuda", dtype=torch.float16), 3,
                             torch.zeros(4, device="cuda"))
    assert e.value.status == bez.Status.UNSUPPORTED


@pytest.mark.parametrize("rational", [False, True])
def test_parameters_next_to_knots_pick_their_span(rational):
    # Degree-1 splines have kinks at every knot: evaluating the neighbouring
    # span a hair outside its interval costs a first-order error there.
    # Sample at the FP32 neighbours of every knot k / (n - p).
    torch = need_gpu()
    rng = np.random.default_rng(700 + rational)
    n, p = 61, 1
    ctrl = rng.uniform(-1, 1, size=(64, n, 3)).astype(np.float32)
    w = rng.uniform(0.5, 2, size=(64, n)).astype(np.float32) if rational else None
    knots = np.array([k / (n - p) for k in range(n - p + 1)], np.float32)
    t = np.unique(np.concatenate([knots, np.nextafter(knots, np.float32(0)), np.nextafter(knots, np.float32(1))]))
    t = t[(t >= 0) & (t <= 1)].astype(np.float32)
    got = _bspline(torch, ctrl, p, t, weights=w)
    ref = oracle.bspline(ctrl, p, t, weights=w)
    assert normalised_error(got, ref).max() <= FP32_BAR
