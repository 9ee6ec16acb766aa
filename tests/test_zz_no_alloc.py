"""The allocation-free spline entry point (bez_eval_spline_noalloc).

Some callers cannot let a library allocate device memory: code that must
never synchronise the device (cudaMalloc and cudaFree can), hosts whose
memory manager owns all device memory, and plugins that may only use the
buffers they are given.  This entry point keeps its span scratch in a fixed
array built into the library.  The test calls it through the C ABI twice in
a row with different inputs (the second call must not see stale spans from
the first) and compares each result with bez_eval_bspline / bez_eval_nurbs,
within the FP32 tolerance the other spline tests use.  The file is named so
that pytest collects it last."""
import numpy as np
import pytest

from gpu_util import need_gpu, normalised_error

pytestmark = pytest.mark.gpu
FP32_BAR = 1e-6


def test_noalloc_matches_allocating_entry_points_twice():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(2026)
    cases = [dict(n=640, n_ctrl=20, p=3, rational=False, n_t=257),
             dict(n=333, n_ctrl=11, p=5, rational=True, n_t=101)]
    for case in cases:
        ctrl = torch.from_numpy(rng.uniform(-1, 1, (case["n"], case["n_ctrl"], 3)).astype(np.float32)).cuda()
        w = (torch.from_numpy(rng.uniform(0.5, 2, (case["n"], case["n_ctrl"])).astype(np.float32)).cuda()
             if case["rational"] else None)
        t = torch.from_numpy(rng.uniform(0, 1, case["n_t"]).astype(np.float32)).cuda()
        out = torch.empty((case["n"], case["n_t"], 3), device="cuda")
        got = bez.bez_eval_spline_noalloc(ctrl, case["p"], t, weights=w, out=out)
        if w is None:
            ref = bez.bez_eval_bspline(ctrl, case["p"], t)
        else:
            ref = bez.bez_eval_nurbs(ctrl, w, case["p"], t)
        torch.cuda.synchronize()
        g, r = got.cpu().numpy(), ref.cpu().numpy().astype(np.float64)
        assert normalised_error(g, r).max() <= FP32_BAR
        assert np.isfinite(g).all()


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
