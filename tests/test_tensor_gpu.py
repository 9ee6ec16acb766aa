"""GPU parity of tensor-product surfaces and volumes (bez_eval_surface /
bez_eval_volume, paper Sec. 2.2) against the oracle's double / triple
Bernstein sums at the FP32 bar (1e-6 of the bounding-box diagonal of the
patch's sampled points; scalar volumes use the control-value range)."""
import numpy as np
import pytest

import oracle
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu
FP32_BAR = 1e-6


def _err_surface(got, ref):
    g = np.asarray(got, np.float64).reshape(ref.shape[0], -1, ref.shape[-1])
    r = ref.reshape(ref.shape[0], -1, ref.shape[-1])
    err = np.linalg.norm(g - r, axis=-1).max(axis=1)
    diag = np.linalg.norm(r.max(axis=1) - r.min(axis=1), axis=-1)
    return err / np.maximum(diag, 2.0 ** -4)


def _err_ctrl(got, ref, ctrl):
    g = np.asarray(got, np.float64).reshape(ref.shape[0], -1, ref.shape[-1])
    r = ref.reshape(ref.shape[0], -1, ref.shape[-1])
    c = np.asarray(ctrl, np.float64).reshape(ctrl.shape[0], -1, ctrl.shape[-1])
    err = np.linalg.norm(g - r, axis=-1).max(axis=1)
    diag = np.linalg.norm(c.max(axis=1) - c.min(axis=1), axis=-1)
    return err / np.maximum(diag, 2.0 ** -4)


def test_bicubic_fast_path():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(1)
    ctrl = rng.uniform(-1, 1, (777, 4, 4, 3)).astype(np.float32)
    got = bez.bez_eval_surface(torch.from_numpy(ctrl).cuda(), 32, 32).cpu().numpy()
    ref = oracle.surface(ctrl, 32, 32)
    assert _err_surface(got, ref).max() <= FP32_BAR
    np.testing.assert_array_equal(got[:, 0, 0], ctrl[:, 0, 0])      # corner interpolation is exact
    np.testing.assert_array_equal(got[:, -1, -1], ctrl[:, -1, -1])


@pytest.mark.parametrize("nu,nv", [(1, 4), (5, 20), (33, 36), (64, 256), (65, 8), (200, 40)])
def test_bicubic_grid_shapes(nu, nv):
    # nu <= 64 takes the warp-per-patch kernel (ragged 32-point row segments
    # when nv is not a multiple of 32), larger nu the block-per-patch kernel
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(nu * 1000 + nv)
    ctrl = rng.uniform(-1, 1, (37, 4, 4, 3)).astype(np.float32)
    got = bez.bez_eval_surface(torch.from_numpy(ctrl).cuda(), nu, nv).cpu().numpy()
    ref = oracle.surface(ctrl, nu, nv)
    assert got.shape == ref.shape
    assert _err_ctrl(got, ref, ctrl).max() <= FP32_BAR
    np.testing.assert_array_equal(got[:, 0, 0], ctrl[:, 0, 0])


@pytest.mark.parametrize("du,dv,dim,nu,nv", [(3, 3, 3, 17, 9), (1, 2, 3, 5, 7), (4, 2, 2, 33, 12), (7, 5, 4, 8, 8),
                                             (3, 3, 1, 32, 32), (2, 6, 3, 1, 1)])
def test_generic_surfaces(du, dv, dim, nu, nv):
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(10 * du + dv)
    ctrl = rng.uniform(-1, 1, (131, du + 1, dv + 1, dim)).astype(np.float32)
    got = bez.bez_eval_surface(torch.from_numpy(ctrl).cuda(), nu, nv).cpu().numpy()
    ref = oracle.surface(ctrl, nu, nv)
    err = _err_surface(got, ref) if dim == 3 and nu * nv > 1 else _err_ctrl(got, ref, ctrl)
    assert err.max() <= FP32_BAR


@pytest.mark.parametrize("du,dv,dw,dim,n", [(3, 3, 3, 1, 16), (2, 3, 1, 3, 5), (1, 1, 1, 4, 9)])
def test_volumes(du, dv, dw, dim, n):
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(100 + du + dv + dw)
    ctrl = rng.normal(size=(97, du + 1, dv + 1, dw + 1, dim)).astype(np.float32)
    got = bez.bez_eval_volume(torch.from_numpy(ctrl).cuda(), n, n, n).cpu().numpy()
    ref = oracle.volume(ctrl, n, n, n)
    assert _err_ctrl(got, ref, ctrl).max() <= FP32_BAR


@pytest.mark.parametrize("nu,nv,nw", [(16, 16, 16), (1, 3, 4), (5, 7, 12), (32, 20, 256), (33, 4, 8), (8, 8, 6)])
def test_tricubic_scalar_volume_shapes(nu, nv, nw):
    # nu <= 32 with nw a multiple of 4 takes the warp-per-volume kernel,
    # the others the block-per-volume kernel; both against the triple sum
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(nu * 10000 + nv * 100 + nw)
    ctrl = rng.normal(size=(41, 4, 4, 4, 1)).astype(np.float32)
    got = bez.bez_eval_volume(torch.from_numpy(ctrl).cuda(), nu, nv, nw).cpu().numpy()
    ref = oracle.volume(ctrl, nu, nv, nw)
    assert got.shape == ref.shape
    assert _err_ctrl(got, ref, ctrl).max() <= FP32_BAR
    np.testing.assert_array_equal(got[:, 0, 0, 0, 0], ctrl[:, 0, 0, 0, 0])   # corner


def test_half_bf16_storage_and_host_arrays():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(7)
    ctrl = rng.uniform(-1, 1, (64, 4, 4, 3)).astype(np.float32)
    for dt in (torch.float16, torch.bfloat16):
        c = torch.from_numpy(ctrl).cuda().to(dt)
        got = bez.bez_eval_surface(c, 32, 32).cpu().numpy()
        ref = oracle.surface(c.float().cpu().numpy(), 32, 32)
        assert _err_surface(got, ref).max() <= FP32_BAR
    host = bez.bez_eval_surface(ctrl, 16, 16)
    dev = bez.bez_eval_surface(torch.from_numpy(ctrl).cuda(), 16, 16).cpu().numpy()
    np.testing.assert_array_equal(host, dev)


def test_tensor_argument_errors():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval_surface(torch.zeros((2, 4, 4, 3), device="cuda"), 300, 4)
    assert e.value.status == bez.Status.UNSUPPORTED
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval_surface(torch.zeros((2, 4, 4, 3), device="cuda"), 4, 4, variant=bez.Variant.TENSOR)
    assert e.value.status == bez.Status.UNSUPPORTED
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval_volume(torch.zeros((2, 4, 4, 4, 1), device="cuda"), 0, 4, 4)
    assert e.value.status == bez.Status.INVALID_ARG
