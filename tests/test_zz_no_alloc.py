"""The allocation-free spline entry point (bez_eval_spline_noalloc).

Some callers cannot let a library allocate device memory: code that must
never synchronise the device (cudaMalloc and cudaFree can), hosts whose
memory manager owns all device memory, and plugins that may only use the
buffers they are given.  This entry point keeps its span scratch in a fixed
array built into the library.  The tests call it through the C ABI several
times in a row with different inputs (a later call must not see stale spans
from an earlier one) and compare each result with the FP64 oracle's
Cox-de Boor evaluation at the FP32 bar the other spline tests use, and with
the allocating entry points on the same inputs.  The file is named so that
pytest collects it last."""
import numpy as np
import pytest

import oracle
from gpu_util import need_gpu, normalised_error

pytestmark = pytest.mark.gpu
FP32_BAR = 1e-6


def _random_knots(rng, B, n, p):
    """Clamped knot vectors with random interior knots on a 1/16 grid
    (interior multiplicity at most p)."""
    U = np.empty((B, n + p + 1), np.float32)
    for b in range(B):
        while True:
            inner = np.sort(rng.integers(1, 16, n - p - 1)) / 16.0
            _, counts = np.unique(inner, return_counts=True)
            if counts.size == 0 or counts.max() <= p:
                break
        U[b] = np.concatenate([np.zeros(p + 1), inner, np.ones(p + 1)])
    return U


def test_noalloc_matches_oracle_and_allocating_entry_points_twice():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(2026)
    cases = [dict(n=640, n_ctrl=20, p=3, rational=False, n_t=257),
             dict(n=333, n_ctrl=11, p=5, rational=True, n_t=101)]
    for case in cases:
        ctrl_np = rng.uniform(-1, 1, (case["n"], case["n_ctrl"], 3)).astype(np.float32)
        w_np = (rng.uniform(0.5, 2, (case["n"], case["n_ctrl"])).astype(np.float32) if case["rational"] else None)
        t_np = rng.uniform(0, 1, case["n_t"]).astype(np.float32)
        ctrl = torch.from_numpy(ctrl_np).cuda()
        w = None if w_np is None else torch.from_numpy(w_np).cuda()
        t = torch.from_numpy(t_np).cuda()
        out = torch.empty((case["n"], case["n_t"], 3), device="cuda")
        got = bez.bez_eval_spline_noalloc(ctrl, case["p"], t, weights=w, out=out)
        if w is None:
            alloc = bez.bez_eval_bspline(ctrl, case["p"], t)
        else:
            alloc = bez.bez_eval_nurbs(ctrl, w, case["p"], t)
        torch.cuda.synchronize()
        g = got.cpu().numpy()
        ref = oracle.bspline(ctrl_np, case["p"], t_np, weights=w_np)
        assert normalised_error(g, ref).max() <= FP32_BAR
        assert normalised_error(alloc.cpu().numpy(), ref).max() <= FP32_BAR
        assert np.isfinite(g).all()


@pytest.mark.parametrize("rational", [False, True])
def test_noalloc_knots_per_curve_t_and_lengths(rational):
    # explicit non-uniform knots (the separately checked knots pointer),
    # per-curve parameters, and the fused polyline-length output
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(2027 + rational)
    B, n, p, n_t = 211, 12, 3, 97
    ctrl_np = rng.uniform(-1, 1, (B, n, 3)).astype(np.float32)
    w_np = rng.uniform(0.5, 2, (B, n)).astype(np.float32) if rational else None
    U_np = _random_knots(rng, B, n, p)
    t_np = np.sort(rng.uniform(0, 1, (B, n_t)).astype(np.float32), axis=1)
    t_np[:, 0] = U_np[:, p + 1]                       # a parameter on an interior knot
    dev = lambda x: None if x is None else torch.from_numpy(x).cuda()
    ctrl, w, U, t = dev(ctrl_np), dev(w_np), dev(U_np), dev(t_np)
    ref = oracle.bspline(ctrl_np, p, t_np, weights=w_np, knots=U_np)
    pts = bez.bez_eval_spline_noalloc(ctrl, p, t, weights=w, knots=U, t_mode=bez.TMode.PER_CURVE)
    L = bez.bez_eval_spline_noalloc(ctrl, p, t, weights=w, knots=U, t_mode=bez.TMode.PER_CURVE,
                                    out_mode=bez.OutMode.POLYLINE_LENGTH)
    if rational:
        L_alloc = bez.bez_eval_nurbs(ctrl, w, p, t, knots=U, t_mode=bez.TMode.PER_CURVE,
                                     out_mode=bez.OutMode.POLYLINE_LENGTH)
    else:
        L_alloc = bez.bez_eval_bspline(ctrl, p, t, knots=U, t_mode=bez.TMode.PER_CURVE,
                                       out_mode=bez.OutMode.POLYLINE_LENGTH)
    torch.cuda.synchronize()
    assert normalised_error(pts.cpu().numpy(), ref).max() <= FP32_BAR
    L_ref = oracle.polyline_length(ref)
    diag = np.maximum(np.linalg.norm(ref.max(axis=1) - ref.min(axis=1), axis=-1), 2.0 ** -4)
    # each of the n_t - 1 segments moves by at most twice the point bar, plus
    # FP32 rounding of the sum
    tol = 2 * (n_t - 1) * FP32_BAR * diag + (n_t + 12) * 2.0 ** -24 * L_ref + 1e-7
    got_L = L.cpu().numpy()
    assert np.all(np.abs(got_L - L_ref) <= tol)
    np.testing.assert_allclose(got_L, L_alloc.cpu().numpy(), rtol=0, atol=float(tol.max()))


def test_noalloc_rejects_oversize_and_host_arrays():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    # 4,194,304 span floats at most: 100,000 cubic 3D curves of 20 points need 20,400,000
    big = torch.zeros((100000, 20, 3), device="cuda")
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval_spline_noalloc(big, 3, torch.zeros(4, device="cuda"))
    assert e.value.status == bez.Status.INVALID_ARG and "16 MiB" in str(e.value)
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval_spline_noalloc(torch.zeros((2, 8, 3)), 3, torch.zeros(4))
    assert e.value.status == bez.Status.INVALID_ARG
