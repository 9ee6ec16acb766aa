"""GPU parity of the adjoint kernel (bez_eval_backward) and the autograd
Function, against the oracle's analytic gradients (which the CPU tests pin
to finite differences and torch's CPU autograd).

Tolerances from the FP32 arithmetic: a per-curve gradient is a sum over
n_t samples of terms each computed with O(d) roundings, accumulated per
lane then by a 5-level butterfly, so |error| <= (n_t/32 + 2d + 12) u
sum_j |term_j|, with sum_j |term_j| taken from the oracle run on |g|.  dL/dt
has no sum; its error is O(d) roundings of g . C'."""
import numpy as np
import pytest

import oracle
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu
U = 2.0 ** -24


def _cuda(torch, x):
    return None if x is None else torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()


def _check(torch, ctrl, t, g, weights=None):
    from paper_2603_15447_gb300 import bez
    gc, gw, gt = bez.bez_eval_backward(_cuda(torch, ctrl), _cuda(torch, t), _cuda(torch, g),
                                       weights=_cuda(torch, weights))
    torch.cuda.synchronize()
    rc, rw, rt = oracle.bezier_grad(ctrl, t, g, weights=weights)
    ac, aw, _ = oracle.bezier_grad(ctrl, t, np.abs(g), weights=weights)     # sum_j |term_j| for the ctrl sums
    B, d1, dim = ctrl.shape
    d = d1 - 1
    n_t = t.shape[-1]
    k = (n_t / 32 + 2 * d + 12) * U
    assert np.all(np.abs(gc.cpu().numpy() - rc) <= k * ac + 1e-30)
    if weights is not None:
        # |P_i - C| <= range of the control points; bound the weight sums the same way
        span = np.abs(ctrl).max() * 2
        aw2 = oracle.bezier_grad(ctrl, t, np.abs(g), weights=weights)[0].sum(axis=2) * span / weights.min()
        assert np.all(np.abs(gw.cpu().numpy() - rw) <= k * aw2 * 4 + 1e-30)
    # dL/dt: scale of g . C'
    if weights is None:
        dmax = d * np.abs(np.diff(ctrl, axis=1)).max()
        scale = np.linalg.norm(g, axis=-1) * dmax * np.sqrt(dim)
    else:
        w = weights
        wp = ctrl * w[:, :, None]
        dmax = d * (np.abs(np.diff(wp, axis=1)).max() + np.abs(ctrl).max() * np.abs(np.diff(w, axis=1)).max())
        scale = np.linalg.norm(g, axis=-1) * dmax * np.sqrt(dim) / w.min()
    if t.ndim == 1:
        # shared t: summed over curves
        tol = (B + 16 * d + 32) * U * scale.sum(axis=0)
    else:
        tol = (16 * d + 32) * U * scale
    assert np.all(np.abs(gt.cpu().numpy() - rt) <= tol + 1e-30)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6, 7, 9])
@pytest.mark.parametrize("rational", [False, True])
def test_adjoint_per_curve_t(d, rational):
    torch = need_gpu()
    rng = np.random.default_rng(10 * d + rational)
    B, n_t = 301, 77
    ctrl = rng.uniform(-1, 1, (B, d + 1, 3)).astype(np.float32)
    w = rng.uniform(0.5, 2, (B, d + 1)).astype(np.float32) if rational else None
    t = rng.uniform(0, 1, (B, n_t)).astype(np.float32)
    t[:, 0] = -0.5                                   # clamped: zero dL/dt
    g = rng.normal(size=(B, n_t, 3)).astype(np.float32)
    _check(torch, ctrl, t, g, w)


@pytest.mark.parametrize("rational", [False, True])
@pytest.mark.parametrize("dim", [1, 2, 4])
def test_adjoint_shared_t_and_dims(rational, dim):
    torch = need_gpu()
    rng = np.random.default_rng(100 + dim + rational)
    B, n_t, d = 257, 40, 3
    ctrl = rng.uniform(-1, 1, (B, d + 1, dim)).astype(np.float32)
    w = rng.uniform(0.5, 2, (B, d + 1)).astype(np.float32) if rational else None
    t = rng.uniform(0, 1, n_t).astype(np.float32)
    g = rng.normal(size=(B, n_t, dim)).astype(np.float32)
    _check(torch, ctrl, t, g, w)


def test_autograd_function_matches_adjoint_and_finite_differences():
    torch = need_gpu()
    from paper_2603_15447_gb300.autograd import bezier_curve
    rng = np.random.default_rng(7)
    ctrl = torch.tensor(rng.uniform(-1, 1, (16, 4, 3)), dtype=torch.float32, device="cuda", requires_grad=True)
    w = torch.tensor(rng.uniform(0.5, 2, (16, 4)), dtype=torch.float32, device="cuda", requires_grad=True)
    t = torch.tensor(rng.uniform(0.1, 0.9, (16, 20)), dtype=torch.float32, device="cuda", requires_grad=True)
    target = torch.tensor(rng.uniform(-1, 1, (16, 20, 3)), dtype=torch.float32, device="cuda")
    loss = ((bezier_curve(ctrl, t, w) - target) ** 2).sum()
    loss.backward()
    rc, rw, rt = oracle.bezier_grad(ctrl.detach().cpu().numpy(), t.detach().cpu().numpy(),
                                    2 * (oracle.bezier(ctrl.detach().cpu().numpy(), t.detach().cpu().numpy(),
                                                       weights=w.detach().cpu().numpy())
                                         - target.cpu().numpy()),
                                    weights=w.detach().cpu().numpy())
    np.testing.assert_allclose(ctrl.grad.cpu().numpy(), rc, rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(w.grad.cpu().numpy(), rw, rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(t.grad.cpu().numpy(), rt, rtol=1e-4, atol=1e-4)
    # central differences through the FP32 forward kernel on a few entries
    eps = 1e-2

    def L(c_, w_, t_):
        with torch.no_grad():
            return float(((bezier_curve(c_, t_, w_) - target) ** 2).sum().double())

    for (i, j, k) in [(0, 0, 0), (3, 2, 1), (15, 3, 2)]:
        e = torch.zeros_like(ctrl)
        e[i, j, k] = eps
        fd = (L(ctrl + e, w, t) - L(ctrl - e, w, t)) / (2 * eps)
        assert abs(fd - float(ctrl.grad[i, j, k])) <= 2e-3 * max(1.0, abs(fd))
    for (i, j) in [(0, 0), (7, 11), (15, 19)]:
        e = torch.zeros_like(t)
        e[i, j] = eps
        fd = (L(ctrl, w, t + e) - L(ctrl, w, t - e)) / (2 * eps)
        assert abs(fd - float(t.grad[i, j])) <= 5e-3 * max(1.0, abs(fd))


def test_adam_fit_reaches_noise_floor():
    # the fitting workload at reduced size: curves fitted to noisy samples of
    # random cubics (sigma 0.01) with Adam (lr 1e-2, 200 steps) through the
    # autograd Function, t clamped to [0,1] after each step
    torch = need_gpu()
    from paper_2603_15447_gb300 import synth
    from paper_2603_15447_gb300.autograd import bezier_curve
    truth, t_true, noise, init = synth.fit(n_curves=2048, n_t=512)
    ref = oracle.bezier(truth, t_true)
    target = torch.tensor((ref + noise).astype(np.float32), device="cuda")
    ctrl = torch.tensor(init, device="cuda", requires_grad=True)
    t = torch.tensor(np.tile((np.arange(512) / 511.0).astype(np.float32), (2048, 1)), device="cuda",
                     requires_grad=True)
    opt = torch.optim.Adam([ctrl, t], lr=1e-2)
    first = None
    for step in range(200):
        opt.zero_grad()
        loss = ((bezier_curve(ctrl, t) - target) ** 2).mean()
        loss.backward()
        opt.step()
        with torch.no_grad():
            t.clamp_(0, 1)
        if first is None:
            first = float(loss)
    final = float(loss)
    assert final < first / 20, (first, final)
    assert np.sqrt(final) < 0.1
