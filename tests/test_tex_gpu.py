"""GPU parity of the texture-path evaluators (paper Sec. 2, 2.3, 4 and Fig. 3).

Linear filtering works with weights of 8 fractional bits (Sec. 2.3), so a
texture evaluator does not reach the oracle to FP32 accuracy.  The tolerance
of one filtered fetch is taken as

    (number of filtered axes) x (2^-8 + 2^-11) x |range of the tile's texels|

per point: the filtered value is a weighted mean of the tile's texels whose
weights still sum to one (measured exactly by the probe below), so moving
weight between texels moves the result by at most the moved weight times the
texel range; each filtered axis moves at most 2^-8 (8-bit weights; the probe
sees up to 1.5 x 2^-8 on one marginal when three axes are off-centre, within
3 x 2^-8) plus 2^-11 for the FP32 rounding of the unnormalised coordinate in
atlases up to 4096 texels wide.  FP32 lerps done afterwards in registers are
convex and do not enlarge the error.  The tiles are rebuilt here from the
paper's layouts.  This is a hardware-model tolerance: the paper fixes the
weight format, not the filter's internal rounding."""
import numpy as np
import pytest

import oracle
from gpu_util import need_gpu, normalised_error

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
WERR = 2.0 ** -8 + 2.0 ** -11


def _run(torch, ctrl, t=None, n_t=None, variant="TEX_DECASTELJAU", out_mode="POINTS", t_mode=None, seed=0,
         stream_id=0, half=False):
    from paper_2603_15447_gb300 import bez
    c = torch.from_numpy(ctrl).cuda()
    if half:
        c = c.half()
    tt = None if t is None else torch.from_numpy(np.ascontiguousarray(t, np.float32)).cuda()
    out = bez.bez_eval(c, tt, n_t=n_t, variant=bez.Variant[variant], out_mode=bez.OutMode[out_mode],
                       t_mode=None if t_mode is None else bez.TMode[t_mode], seed=seed, stream_id=stream_id)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _range(tiles):
    """|max - min|_2 over the texels of each tile: tiles [B][n_texels][dim]."""
    return np.linalg.norm(tiles.max(axis=1) - tiles.min(axis=1), axis=-1)


def _seiler_terms(b):
    d = b.shape[1] - 1
    from math import comb
    d1 = d * (b[:, 1] - b[:, 0]) - (b[:, d] - b[:, 0])
    dl = d * (b[:, d - 1] - b[:, d]) - (b[:, 0] - b[:, d])
    if d >= 4:
        d2 = (comb(d, 2) * (b[:, 2] - b[:, 1]) - comb(d - 2, 2) * (b[:, 1] - b[:, 0])
              - (d - 3) * (b[:, d - 1] - b[:, d]) - 3 * (b[:, d - 1] - b[:, 1]))
        dl2 = (comb(d, 2) * (b[:, d - 2] - b[:, d - 1]) - comb(d - 2, 2) * (b[:, d - 1] - b[:, d])
               - (d - 3) * (b[:, 1] - b[:, 0]) - 3 * (b[:, 1] - b[:, d - 1]))
    else:
        d2 = dl2 = np.zeros_like(d1)
    return d1, dl, d2, dl2


def texture_bound(variant, ctrl, texel_eps=U):
    """Per-curve bound on |P_tex - C| (see module doc).  texel_eps: relative
    rounding of a stored texel (2^-24 float, 2^-11 half)."""
    b = ctrl.astype(np.float64)
    B, d1_, dim = b.shape
    d = d1_ - 1
    if variant == "TEX_DECASTELJAU":
        # tile of window i holds b_i..b_(i+3) (degree <= 2: b_0..b_d)
        w = min(d, 3)
        bound = np.max([_range(b[:, i:i + w + 1]) for i in range(d - w + 1)], axis=0) * w * WERR
        tex_mag = np.abs(b).max(axis=(1, 2))
    elif variant == "TEX_HYBRID":
        w = min(d, 2)
        bound = np.max([_range(b[:, i:i + w + 1]) for i in range(d - w + 1)], axis=0) * w * WERR
        tex_mag = np.abs(b).max(axis=(1, 2))
    else:
        d1, dl, d2, dl2 = _seiler_terms(b)
        b0, bd = b[:, 0], b[:, d]
        s1, s2 = b0 + d1, bd + dl
        if d <= 3:
            tiles = np.stack([b0, bd, s1, s2], 1)
            axes = 2
        else:
            tiles = np.stack([b0, bd, s1, s2, s1 + d2, s2 + dl2], 1)
            axes = 3
        bound = axes * WERR * _range(tiles)
        tex_mag = np.abs(tiles).max(axis=(1, 2))
    # texel rounding (Seiler sums, half texels), filter and register-lerp rounding
    slack = (4 * texel_eps + (d + 12) * U) * tex_mag * np.sqrt(dim)
    return bound + slack


def test_filter_weight_probe_single_axis():
    # Along one axis (the others at texel centres) the weight is the
    # fractional coordinate on 8 fractional bits (Sec. 2.3), within 2^-8 of
    # exact and exact at texel centres; weights sum to one.
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    k = np.arange(0, 4097)
    frac = k / 4096.0
    xyz = np.stack([0.5 + frac, np.full_like(frac, 0.5), np.full_like(frac, 1.5)], 1).astype(np.float32)
    got = bez.bez_probe_filter(torch.from_numpy(xyz).cuda()).cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(got[:, 0] * 256, np.round(got[:, 0] * 256))
    assert np.abs(got[:, 0] - frac).max() <= 2.0 ** -8
    np.testing.assert_array_equal(got[:, 1], 0.0)
    np.testing.assert_array_equal(got[:, 2], 1.0)
    np.testing.assert_array_equal(got[:, 3], 1.0)
    assert got[0, 0] == 0.0 and got[-1, 0] == 1.0
    # three axes off-centre: weights still sum to one, every marginal within
    # the 3 x 2^-8 the tolerance above allows for a trilinear fetch
    g = np.arange(0, 33) / 32.0
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([0.5 + X.ravel(), 0.5 + Y.ravel(), 0.5 + Z.ravel()], 1).astype(np.float32)
    got3 = bez.bez_probe_filter(torch.from_numpy(xyz).cuda()).cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(got3[:, 3], 1.0)
    for ax, E in enumerate((X, Y, Z)):
        assert np.abs(got3[:, ax] - E.ravel()).max() <= 3 * 2.0 ** -8
    err = got[:, 0] - frac
    mode = "round-to-nearest" if err.min() < -2.0 ** -10 else "truncate"
    print(f"\nsingle-axis filter weight: 8 fractional bits, {mode}; max |w - t| = {np.abs(err).max():.6f}")


@pytest.mark.parametrize("variant,d", [("TEX_DECASTELJAU", d) for d in (1, 2, 3, 4, 5, 7)]
                         + [("TEX_HYBRID", d) for d in (1, 2, 3, 4, 6)]
                         + [("TEX_SEILER", d) for d in (2, 3, 4, 5)])
def test_texture_points_within_weight_bound(variant, d):
    torch = need_gpu()
    rng = np.random.default_rng(40 + d)
    ctrl = rng.uniform(-1, 1, size=(1001, d + 1, 3)).astype(np.float32)
    t = rng.uniform(0, 1, 71).astype(np.float32)
    got = _run(torch, ctrl, t, variant=variant)
    ref = oracle.bezier(ctrl, t)
    err = np.linalg.norm(got - ref, axis=-1).max(axis=1)
    bound = texture_bound(variant, ctrl)
    assert np.all(err <= bound), (err / bound).max()
    print(f"\n{variant} d={d}: max normalised error {normalised_error(got, ref).max():.3g}, "
          f"max error / bound {(err / bound).max():.3f}")


@pytest.mark.parametrize("variant", ["TEX_DECASTELJAU", "TEX_HYBRID", "TEX_SEILER"])
def test_texture_endpoints_exact_and_nan(variant):
    torch = need_gpu()
    rng = np.random.default_rng(50)
    ctrl = rng.uniform(-1, 1, size=(300, 4, 3)).astype(np.float32)
    got = _run(torch, ctrl, np.array([0.0, 1.0, -1.0, 2.0, np.nan], np.float32), variant=variant)
    np.testing.assert_array_equal(got[:, 0], ctrl[:, 0])
    np.testing.assert_array_equal(got[:, 1], ctrl[:, 3])
    np.testing.assert_array_equal(got[:, 2], ctrl[:, 0])
    np.testing.assert_array_equal(got[:, 3], ctrl[:, 3])
    assert np.isnan(got[:, 4]).all()


@pytest.mark.parametrize("variant", ["TEX_DECASTELJAU", "TEX_HYBRID", "TEX_SEILER"])
def test_texture_dims_modes_and_half_texels(variant):
    torch = need_gpu()
    rng = np.random.default_rng(60)
    for dim in (1, 2, 4):
        ctrl = rng.uniform(-1, 1, size=(257, 4, dim)).astype(np.float32)
        t = rng.uniform(0, 1, (257, 40)).astype(np.float32)
        got = _run(torch, ctrl, t, variant=variant, t_mode="PER_CURVE")
        err = np.linalg.norm(got - oracle.bezier(ctrl, t), axis=-1).max(axis=1)
        assert np.all(err <= texture_bound(variant, ctrl))
    ctrl = rng.uniform(-1, 1, size=(300, 4, 3)).astype(np.float32)
    got = _run(torch, ctrl, n_t=64, variant=variant, t_mode="UNIFORM")
    err = np.linalg.norm(got - oracle.bezier_grid(ctrl, 64), axis=-1).max(axis=1)
    assert np.all(err <= texture_bound(variant, ctrl))
    got = _run(torch, ctrl, n_t=50, variant=variant, t_mode="HASH", seed=3, stream_id=9)
    err = np.linalg.norm(got - oracle.bezier(ctrl, oracle.hash_t(3, 9, 0, 300, 50)), axis=-1).max(axis=1)
    assert np.all(err <= texture_bound(variant, ctrl))
    # half4 texels: the control points the kernel sees are the FP16 values
    stored = ctrl.astype(np.float16).astype(np.float32)
    t = rng.uniform(0, 1, 33).astype(np.float32)
    got = _run(torch, ctrl, t, variant=variant, half=True)
    err = np.linalg.norm(got - oracle.bezier(stored, t), axis=-1).max(axis=1)
    assert np.all(err <= texture_bound(variant, stored, texel_eps=2.0 ** -11))


@pytest.mark.parametrize("variant", ["TEX_DECASTELJAU", "TEX_HYBRID", "TEX_SEILER"])
def test_texture_polyline_length(variant):
    torch = need_gpu()
    rng = np.random.default_rng(70)
    n, n_t = 500, 1024
    ctrl = rng.uniform(-1, 1, size=(n, 4, 3)).astype(np.float32)
    got = _run(torch, ctrl, n_t=n_t, variant=variant, out_mode="POLYLINE_LENGTH", t_mode="HASH", seed=11,
               stream_id=2)
    pts = oracle.bezier(ctrl, oracle.hash_t(11, 2, 0, n, n_t))
    L = oracle.polyline_length(pts)
    tol = 2 * (n_t - 1) * texture_bound(variant, ctrl) + (n_t / 32 + 12) * U * L
    assert np.all(np.abs(got - L) <= tol)


def test_texture_unsupported_combinations():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval(torch.zeros((4, 7, 3), device="cuda"), torch.zeros(3, device="cuda"),
                     variant=bez.Variant.TEX_SEILER)
    assert e.value.status == bez.Status.UNSUPPORTED
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval(torch.zeros((4, 4, 3), device="cuda", dtype=torch.bfloat16), torch.zeros(3, device="cuda"),
                     variant=bez.Variant.TEX_DECASTELJAU)
    assert e.value.status == bez.Status.UNSUPPORTED
