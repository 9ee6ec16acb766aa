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


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("n_t", [4, 132, 260, 512])
def test_adjoint_low_degrees_and_sample_counts(d, n_t):
    # integral 3D curves with per-curve t over sample counts that are and are
    # not multiples of the 64 samples a warp takes per iteration (a partial
    # last pair); also without dL/dt
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(500 + 10 * d + n_t)
    B = 77
    ctrl = rng.uniform(-1, 1, (B, d + 1, 3)).astype(np.float32)
    t = rng.uniform(0, 1, (B, n_t)).astype(np.float32)
    t[:, 1] = 1.5                                    # clamped: zero dL/dt
    g = rng.normal(size=(B, n_t, 3)).astype(np.float32)
    _check(torch, ctrl, t, g)
    gc, _, gt = bez.bez_eval_backward(_cuda(torch, ctrl), _cuda(torch, t), _cuda(torch, g), need_t=False)
    torch.cuda.synchronize()
    assert gt is None
    rc, _, _ = oracle.bezier_grad(ctrl, t, g)
    ac, _, _ = oracle.bezier_grad(ctrl, t, np.abs(g))
    assert np.all(np.abs(gc.cpu().numpy() - rc) <= (n_t / 32 + 2 * d + 12) * U * ac + 1e-30)


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
    # random cubics (sigma 0.01) through the autograd Function, from random
    # control points and uniformly spaced t.  Adam with its own rate for the
    # control points (5e-2) and for t (1e-3), both decayed on a cosine to 1 %
    # over 500 steps, t clamped to [0, 1] after each step -- the schedule of
    # the benchmark's convergence check.  The RMS residual must come down to the
    # noise level (free t absorb the noise along the curve, so it may end a
    # little below sigma); test_adam_trajectory_matches_oracle_steps checks
    # the individual steps against the oracle.
    torch = need_gpu()
    import math
    from paper_2603_15447_gb300 import synth
    from paper_2603_15447_gb300.autograd import bezier_curve
    sigma, steps, lr = 0.01, 500, (5e-2, 1e-3)
    truth, t_true, noise, init = synth.fit(n_curves=2048, n_t=512, sigma=sigma)
    ref = oracle.bezier(truth, t_true)
    target = torch.tensor((ref + noise).astype(np.float32), device="cuda")
    ctrl = torch.tensor(init, device="cuda", requires_grad=True)
    t = torch.tensor(np.tile((np.arange(512) / 511.0).astype(np.float32), (2048, 1)), device="cuda",
                     requires_grad=True)
    opt = torch.optim.Adam([{"params": [ctrl], "lr": lr[0]}, {"params": [t], "lr": lr[1]}])
    first = None
    for k in range(steps):
        f = 0.01 + 0.99 * 0.5 * (1.0 + math.cos(math.pi * k / steps))
        for g, base in zip(opt.param_groups, lr):
            g["lr"] = base * f
        opt.zero_grad()
        loss = ((bezier_curve(ctrl, t) - target) ** 2).mean()
        loss.backward()
        opt.step()
        with torch.no_grad():
            t.clamp_(0, 1)
        if first is None:
            first = float(loss.detach())
    rms = float(loss.detach()) ** 0.5
    assert first ** 0.5 > 30 * sigma, first
    assert 0.7 * sigma < rms < 1.2 * sigma, rms


def _adam_fp64(theta, g, m, v, k, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1) in FP64; k counts from 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** k)
    vh = v / (1 - b2 ** k)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def test_adam_trajectory_matches_oracle_steps():
    # ten steps of the fused fit step (bez_mse_grad + torch Adam on the GPU)
    # against the same steps driven on the CPU by the oracle's curve and
    # analytic gradient with an FP64 Adam: parameters stay within 1e-4 while
    # each step moves them by up to lr = 1e-2 (a wrong term in a gradient
    # shows up at the step size)
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez, synth
    truth, t_true, noise, init = synth.fit(n_curves=64, n_t=512)
    y = (oracle.bezier(truth, t_true) + noise).astype(np.float32)
    n_c, n_t = y.shape[0], y.shape[1]
    t0 = np.tile((np.arange(n_t) / (n_t - 1.0)).astype(np.float32), (n_c, 1))
    scale = 1.0 / (n_c * n_t * 3)
    ctrl = torch.tensor(init, device="cuda")
    t = torch.tensor(t0, device="cuda")
    target = torch.tensor(y, device="cuda")
    opt = torch.optim.Adam([ctrl, t], lr=1e-2)
    P, T = init.astype(np.float64), t0.astype(np.float64)
    mP, vP, mT, vT = (np.zeros_like(P), np.zeros_like(P), np.zeros_like(T), np.zeros_like(T))
    for k in range(1, 11):
        _, gc, _, gt = bez.bez_mse_grad(ctrl, t, target, loss_scale=scale)
        ctrl.grad, t.grad = gc, gt
        opt.step()
        t.clamp_(0, 1)
        C = oracle.bezier(P, T)
        rc, _, rt = oracle.bezier_grad(P, T, 2 * scale * (C - y))
        P, mP, vP = _adam_fp64(P, rc, mP, vP, k)
        T, mT, vT = _adam_fp64(T, rt, mT, vT, k)
        T = np.clip(T, 0.0, 1.0)
    torch.cuda.synchronize()
    dP = np.abs(ctrl.cpu().numpy() - P).max()
    dT = np.abs(t.cpu().numpy() - T).max()
    assert dP <= 1e-4 and dT <= 1e-4, (dP, dT)
    moved = np.abs(P - init).max()
    assert moved > 0.05, moved                                # the parameters did move


def _dmax_over_wmin(ctrl, w):
    # bound on |C'(t)|: d max|q_(i+1) - q_i| over the homogeneous points, / min w
    d = ctrl.shape[1] - 1
    if w is None:
        return d * np.abs(np.diff(ctrl.astype(np.float64), axis=1)).max()
    wp = ctrl * w[:, :, None]
    return d * (np.abs(np.diff(wp, axis=1)).max() + np.abs(ctrl).max() * np.abs(np.diff(w, axis=1)).max()) / w.min()


@pytest.mark.parametrize("d,rational,shared", [(3, False, False), (5, True, False), (2, False, True), (7, True, True)])
def test_fused_squared_error_step(d, rational, shared):
    # bez_mse_grad: loss s sum ||C - y||^2 and the adjoint of g = 2 s (C - y),
    # against the FP64 oracle.  The kernel's C (Bernstein triangle, then A / W)
    # is within eps_C = (4d + 16) u max|P| of the exact value, which moves
    # each g_j by at most 2 s eps_C per coordinate; on top of that come the
    # adjoint's own sum roundings (module doc).  The per-curve weights
    # w_i B_i / W of dL/dP sum to 1, so over n_t samples the moved g shifts
    # dL/dP by at most n_t 2 s eps_C.
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(700 + d + 10 * rational + 100 * shared)
    B, n_t, dim = 203, 96, 3
    ctrl = rng.uniform(-1, 1, (B, d + 1, dim)).astype(np.float32)
    w = rng.uniform(0.5, 2, (B, d + 1)).astype(np.float32) if rational else None
    t = rng.uniform(0, 1, n_t if shared else (B, n_t)).astype(np.float32)
    C = oracle.bezier(ctrl, t, weights=w) if w is not None else oracle.bezier(ctrl, t)
    y = (C + rng.normal(scale=0.05, size=C.shape)).astype(np.float32)
    s = 1.0 / (B * n_t * dim)
    loss, gc, gw, gt = bez.bez_mse_grad(_cuda(torch, ctrl), _cuda(torch, t), _cuda(torch, y),
                                        weights=_cuda(torch, w), loss_scale=s)
    torch.cuda.synchronize()
    r = C - y.astype(np.float64)
    g = 2 * s * r
    loss_ref = s * (r ** 2).sum(axis=(1, 2))
    rc, rw, rt = oracle.bezier_grad(ctrl, t, g, weights=w)
    ac, _, _ = oracle.bezier_grad(ctrl, t, np.abs(g), weights=w)
    eps_c = (4 * d + 16) * U * np.abs(ctrl).max(axis=(1, 2)).astype(np.float64)   # [B]
    dg = 2 * s * eps_c * (1 + 4 * U)                                             # [B], per coordinate
    k = (n_t / 32 + 2 * d + 12) * U
    lo = loss.cpu().numpy()
    assert lo.shape == (B,)
    assert np.all(np.abs(lo - loss_ref)
                  <= s * (2 * np.abs(r).sum(axis=(1, 2)) * eps_c + n_t * dim * eps_c ** 2) + k * 2 * loss_ref + 1e-30)
    dgc = (n_t * dg)[:, None, None]
    assert np.all(np.abs(gc.cpu().numpy() - rc) <= dgc + k * (ac + dgc) + 1e-30)
    cp = _dmax_over_wmin(ctrl, w) * np.sqrt(dim)
    gmag = np.linalg.norm(g, axis=-1) + np.sqrt(dim) * dg[:, None]             # [B][n_t]
    tol_t = (16 * d + 32) * U * gmag * cp + np.sqrt(dim) * dg[:, None] * cp
    if shared:
        assert np.all(np.abs(gt.cpu().numpy() - rt) <= tol_t.sum(axis=0) * (1 + B * U) + 1e-30)
    else:
        assert np.all(np.abs(gt.cpu().numpy() - rt) <= tol_t + 1e-30)
    if w is None:
        assert gw is None
    else:
        span = np.abs(ctrl).max() * 2
        aw2 = oracle.bezier_grad(ctrl, t, np.abs(g) + dg[:, None, None], weights=w)[0].sum(axis=2) * span / w.min()
        assert np.all(np.abs(gw.cpu().numpy() - rw) <= k * aw2 * 4 + n_t * dim * dg[:, None] * span / w.min() + 1e-30)


def test_fused_step_matches_backward_with_kernel_residual():
    # the fused path is the unfused adjoint fed its own residual: with g formed
    # from the forward kernel's points, the two agree to the FP32 evaluation
    # difference of the two kernels, far inside the oracle tolerances above.
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(77)
    B, n_t, d = 64, 130, 3
    ctrl = torch.from_numpy(rng.uniform(-1, 1, (B, d + 1, 3)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.uniform(0, 1, (B, n_t)).astype(np.float32)).cuda()
    y = torch.from_numpy(rng.uniform(-1, 1, (B, n_t, 3)).astype(np.float32)).cuda()
    loss, gc, _, gt = bez.bez_mse_grad(ctrl, t, y, loss_scale=0.5)
    pts = bez.bez_eval(ctrl, t, variant=bez.Variant.BERNSTEIN)
    g = 2 * 0.5 * (pts - y)
    gc2, _, gt2 = bez.bez_eval_backward(ctrl, t, g)
    torch.cuda.synchronize()
    assert torch.allclose(loss, 0.5 * ((pts - y) ** 2).sum(dim=(1, 2)), rtol=1e-5, atol=1e-6)
    assert torch.allclose(gc, gc2, rtol=1e-4, atol=1e-5)
    assert torch.allclose(gt, gt2, rtol=1e-4, atol=1e-5)


def test_fused_step_host_arrays_match_device():
    # host (NumPy) arguments are staged through the context's buffers; the
    # results equal the device-array call bit for bit
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(78)
    B, n_t, d = 37, 70, 3
    ctrl = rng.uniform(-1, 1, (B, d + 1, 3)).astype(np.float32)
    w = rng.uniform(0.5, 2, (B, d + 1)).astype(np.float32)
    t = rng.uniform(0, 1, (B, n_t)).astype(np.float32)
    y = rng.uniform(-1, 1, (B, n_t, 3)).astype(np.float32)
    host = bez.bez_mse_grad(ctrl, t, y, weights=w, loss_scale=0.25, sync=True)
    dev = bez.bez_mse_grad(_cuda(torch, ctrl), _cuda(torch, t), _cuda(torch, y), weights=_cuda(torch, w),
                           loss_scale=0.25)
    torch.cuda.synchronize()
    for h, g in zip(host, dev):
        assert isinstance(h, np.ndarray)
        np.testing.assert_array_equal(h, g.cpu().numpy())


def test_fused_step_edge_sizes_and_errors():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(79)
    ctrl = _cuda(torch, rng.uniform(-1, 1, (5, 4, 3)).astype(np.float32))
    # no samples: zero loss and zero gradients
    empty_t, empty_y = torch.zeros((5, 0), device="cuda"), torch.zeros((5, 0, 3), device="cuda")
    loss, gc, _, gt = bez.bez_mse_grad(ctrl, empty_t, empty_y, loss_scale=1.0)
    torch.cuda.synchronize()
    assert loss.shape == (5,) and float(loss.abs().max()) == 0.0
    assert float(gc.abs().max()) == 0.0 and gt.numel() == 0
    # no curves: nothing to do
    none_t, none_y = torch.zeros((0, 8), device="cuda"), torch.zeros((0, 8, 3), device="cuda")
    loss, gc, _, _ = bez.bez_mse_grad(ctrl[:0].contiguous(), none_t, none_y)
    assert loss.numel() == 0 and gc.numel() == 0
    # a missing target is rejected before any launch
    import ctypes

    from paper_2603_15447_gb300.bez import Opts, _ptr, context, lib
    o = Opts(int(bez.Variant.AUTO), 0, int(bez.OutMode.POINTS), int(bez.TMode.PER_CURVE), 0, 0, 1, None, 0, 0)
    t = torch.zeros((5, 8), device="cuda")
    gcb = torch.empty((5, 4, 3), device="cuda")
    L = lib()
    if not getattr(L, "_mse_ready", False):
        bez.bez_mse_grad(ctrl, t, torch.zeros((5, 8, 3), device="cuda"))   # sets the argtypes
    st = L.bez_mse_grad(context(0).handle, _ptr(ctrl), None, 5, 3, 3, _ptr(t), 8, None, ctypes.c_float(1.0), None,
                        _ptr(gcb), None, None, ctypes.byref(o), None)
    assert st == int(bez.Status.INVALID_ARG)
