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
         stream_id=0, half=False, tex_share=0, tex_format="AUTO"):
    from paper_2603_15447_gb300 import bez
    c = torch.from_numpy(ctrl).cuda()
    if half:
        c = c.half()
    tt = None if t is None else torch.from_numpy(np.ascontiguousarray(t, np.float32)).cuda()
    out = bez.bez_eval(c, tt, n_t=n_t, variant=bez.Variant[variant], out_mode=bez.OutMode[out_mode],
                       t_mode=None if t_mode is None else bez.TMode[t_mode], seed=seed, stream_id=stream_id,
                       tex_share=tex_share, tex_format=bez.TexFormat[tex_format])
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


def _seiler_terms_peeled(b):
    """lo[k] = d_k, hi[k] = d_(d-k), k = 0..3, by FP64 polynomial division:
    P_0 = C, P_(k+1) = (P_k - L(P_k(0), P_k(1), t)) / (t (1 - t)) (power basis,
    numpy); b [B][d+1][dim]."""
    from math import comb
    B, d1_, dim = b.shape
    d = d1_ - 1
    lo = np.zeros((4, B, dim))
    hi = np.zeros((4, B, dim))
    for c in range(B):
        for a in range(dim):
            # power-basis coefficients, highest degree first
            P = np.zeros(d + 1)
            for i in range(d + 1):
                term = np.poly1d([1.0])
                term = term * comb(d, i) * np.poly1d([-1.0, 1.0]) ** (d - i) * np.poly1d([1.0, 0.0]) ** i
                P = np.polyadd(P, term.coeffs * b[c, i, a])
            P = np.poly1d(P)
            for k in range(4):
                l0, h0 = P(0.0), P(1.0)
                lo[k, c, a], hi[k, c, a] = l0, h0
                if P.order < 2:
                    if k < 3:
                        lo[k + 1:, c, a] = 0.0
                        hi[k + 1:, c, a] = 0.0
                    break
                num = P - np.poly1d([h0 - l0, l0])
                P, _ = np.polydiv(num, np.poly1d([-1.0, 1.0, 0.0]))
    return lo, hi


def texture_bound(variant, ctrl, texel_eps=U, texel_q=0.0):
    """Per-curve bound on |P_tex - C| (see module doc).  texel_eps: relative
    rounding of a stored texel (2^-24 float, 2^-11 half); texel_q: rounding
    of a unorm texel as a fraction of its tile's range (half a code)."""
    b = ctrl.astype(np.float64)
    B, d1_, dim = b.shape
    d = d1_ - 1
    if variant == "TEX_DECASTELJAU":
        # tile of window i holds b_i..b_(i+3) (degree <= 2: b_0..b_d)
        w = min(d, 3)
        R = np.max([_range(b[:, i:i + w + 1]) for i in range(d - w + 1)], axis=0)
        bound = R * (w * WERR + texel_q)
        tex_mag = np.abs(b).max(axis=(1, 2))
    elif variant == "TEX_HYBRID":
        w = min(d, 2)
        R = np.max([_range(b[:, i:i + w + 1]) for i in range(d - w + 1)], axis=0)
        bound = R * (w * WERR + texel_q)
        tex_mag = np.abs(b).max(axis=(1, 2))
    elif d >= 6:
        # degree 6, 7 tile: corners L0, L0 + L1/4, L0 + L2/16, L0 + L1/4 + L2/16 + L3/64
        lo, hi = _seiler_terms_peeled(b)
        c0 = lo[0], hi[0]
        c1 = lo[0] + lo[1] / 4, hi[0] + hi[1] / 4
        c2 = lo[0] + lo[2] / 16, hi[0] + hi[2] / 16
        c3 = c1[0] + lo[2] / 16 + lo[3] / 64, c1[1] + hi[2] / 16 + hi[3] / 64
        tiles = np.stack([*c0, *c1, *c2, *c3], 1)
        bound = (3 * WERR + texel_q) * _range(tiles)
        tex_mag = np.abs(tiles).max(axis=(1, 2))
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
        bound = (axes * WERR + texel_q) * _range(tiles)
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
                         + [("TEX_SEILER", d) for d in (2, 3, 4, 5, 6, 7)])
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
        bez.bez_eval(torch.zeros((4, 9, 3), device="cuda"), torch.zeros(3, device="cuda"),
                     variant=bez.Variant.TEX_SEILER)
    assert e.value.status == bez.Status.UNSUPPORTED
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval(torch.zeros((4, 4, 3), device="cuda", dtype=torch.bfloat16), torch.zeros(3, device="cuda"),
                     variant=bez.Variant.TEX_DECASTELJAU)
    assert e.value.status == bez.Status.UNSUPPORTED


@pytest.mark.parametrize("variant", ["TEX_DECASTELJAU", "TEX_SEILER"])
@pytest.mark.parametrize("dim,nu,nv,half", [(3, 32, 32, False), (1, 5, 20, False), (2, 64, 256, False),
                                            (4, 17, 9, False), (3, 1, 1, False), (3, 32, 32, True)])
def test_texture_bicubic_surface(variant, dim, nu, nv, half):
    # Sec. 2.2: a 2x2x2 RGBA tile per coordinate holds the four column cubics
    # C[.][j][k]; one trilinear read at (u,u,u) gives the isoline control
    # points of row u and the cubic in v runs in FP32.  The v stage is a convex
    # combination, so the error is that of one 3-axis filtered read of the
    # column tile: 3 x WERR x the largest column range of the coordinate.
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(7000 + 100 * dim + nu + nv)
    ctrl = rng.uniform(-1, 1, (301, 4, 4, dim)).astype(np.float32)
    c = torch.from_numpy(ctrl).cuda()
    if half:
        c = c.half()
    got = bez.bez_eval_surface(c, nu, nv, variant=bez.Variant[variant]).cpu().numpy().astype(np.float64)
    src = c.float().cpu().numpy()
    ref = oracle.surface(src, nu, nv)
    if variant == "TEX_DECASTELJAU":
        col_range = (src.max(axis=1) - src.min(axis=1)).max(axis=1)        # [n][dim]: max over columns j
        axes, mag = 3, np.abs(src).max(axis=(1, 2))
    else:
        # the column's 2x2 Seiler tile (Sec. 4 cubic layout), per channel j
        b = src.astype(np.float64)                                         # [n][i][j][k]
        d1 = 3 * (b[:, 1] - b[:, 0]) - (b[:, 3] - b[:, 0])
        d2 = 3 * (b[:, 2] - b[:, 3]) - (b[:, 0] - b[:, 3])
        tile = np.stack([b[:, 0], b[:, 3], b[:, 0] + d1, b[:, 3] + d2], 1)  # [n][4][j][k]
        col_range = (tile.max(axis=1) - tile.min(axis=1)).max(axis=1)
        axes, mag = 2, np.abs(tile).max(axis=(1, 2))
    tol = axes * WERR * col_range + 8 * U * mag                           # [n][dim]
    if half:
        ref_true = oracle.surface(ctrl, nu, nv)
        err_true = np.abs(got - ref_true).max()
        assert err_true <= (axes * WERR * col_range.max() + 2.0 ** -10 * max(1.0, mag.max()))
    err = np.abs(got - ref)                                                # [n][nu][nv][dim]
    assert np.all(err <= tol[:, None, None, :])
    if not half:
        np.testing.assert_array_equal(got[:, 0, 0], ctrl[:, 0, 0])         # texel centres: exact corners
        if nu > 1 and nv > 1:
            np.testing.assert_array_equal(got[:, -1, -1], ctrl[:, -1, -1])


@pytest.mark.parametrize("variant", ["TEX_DECASTELJAU", "TEX_SEILER"])
@pytest.mark.parametrize("fmt", ["AUTO", "UNORM16"])
def test_texture_surface_warps_loop_over_patches(variant, fmt):
    # With at most 32 rows a warp issues the filtered reads of its next patch
    # before sweeping the current one.  20,001 patches on a 5 x 3 grid is more
    # than the resident warps (8 a block x 4 blocks an SM x the SM count), so
    # every warp handles several patches and uses the prefetched rows; each
    # patch is checked against the oracle at the tolerance of the tests above.
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    n = 20001
    assert n > 8 * 4 * n_sm
    rng = np.random.default_rng(7300 + (fmt == "AUTO"))
    ctrl = rng.uniform(-1, 1, (n, 4, 4, 3)).astype(np.float32)
    got = bez.bez_eval_surface(torch.from_numpy(ctrl).cuda(), 5, 3, variant=bez.Variant[variant],
                               tex_format=bez.TexFormat[fmt]).cpu().numpy().astype(np.float64)
    ref = oracle.surface(ctrl, 5, 3)
    b = ctrl.astype(np.float64)
    if variant == "TEX_DECASTELJAU":
        tiles = b                                                          # [n][i][j][k]
        axes = 3
    else:
        d1 = 3 * (b[:, 1] - b[:, 0]) - (b[:, 3] - b[:, 0])
        d2 = 3 * (b[:, 2] - b[:, 3]) - (b[:, 0] - b[:, 3])
        tiles = np.stack([b[:, 0], b[:, 3], b[:, 0] + d1, b[:, 3] + d2], 1)
        axes = 2
    col_range = (tiles.max(axis=1) - tiles.min(axis=1)).max(axis=1)        # [n][dim]
    mag = np.abs(tiles).max(axis=(1, 2))
    q = 2.0 ** -17 if fmt == "UNORM16" else 0.0                             # half a code of the tile's range
    tol = axes * WERR * col_range + q * col_range + 8 * U * mag
    assert np.all(np.abs(got - ref) <= tol[:, None, None, :])


@pytest.mark.parametrize("variant", ["TEX_DECASTELJAU", "TEX_SEILER"])
@pytest.mark.parametrize("fmt,levels", [("UNORM16", 65535.0), ("UNORM8", 255.0)])
@pytest.mark.parametrize("dim,nu,nv", [(3, 32, 32), (1, 7, 19), (4, 64, 5)])
def test_texture_surface_unorm(variant, fmt, levels, dim, nu, nv):
    # unorm tiles: per tile and channel (column cubic j of coordinate k) the
    # texels are stored as codes of (v - lo) / scale with lo, scale the
    # channel's minimum and range over the tile, mapped back after filtering.
    # Rounding to the nearest code moves a texel by at most scale / (2 levels);
    # filtering and the v cubic are convex combinations, so the error bound of
    # the float tiles grows by half a code of the largest channel range.
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(7100 + 10 * dim + nu + int(levels))
    ctrl = rng.uniform(-1, 1, (211, 4, 4, dim)).astype(np.float32)
    ctrl[5] = 0.25                                                        # constant patch: every channel flat
    ctrl[6, :, 2, :] = -0.5                                               # one flat column cubic
    got = bez.bez_eval_surface(torch.from_numpy(ctrl).cuda(), nu, nv, variant=bez.Variant[variant],
                               tex_format=bez.TexFormat[fmt]).cpu().numpy().astype(np.float64)
    ref = oracle.surface(ctrl, nu, nv)
    b = ctrl.astype(np.float64)                                           # [n][i][j][k]
    if variant == "TEX_DECASTELJAU":
        tile = b
        axes = 3
    else:
        d1 = 3 * (b[:, 1] - b[:, 0]) - (b[:, 3] - b[:, 0])
        d2 = 3 * (b[:, 2] - b[:, 3]) - (b[:, 0] - b[:, 3])
        tile = np.stack([b[:, 0], b[:, 3], b[:, 0] + d1, b[:, 3] + d2], 1)
        axes = 2
    col_range = (tile.max(axis=1) - tile.min(axis=1)).max(axis=1)         # [n][dim]
    mag = np.abs(tile).max(axis=(1, 2))
    tol = (axes * WERR + 0.5 / levels) * col_range + 8 * U * mag
    err = np.abs(got - ref)
    assert np.all(err <= tol[:, None, None, :])
    # a flat channel is stored as code 0 with lo = its value: exact up to the FP32 v stage
    assert np.abs(got[5] - 0.25).max() <= 8 * U


@pytest.mark.parametrize("variant", ["TEX_DECASTELJAU", "TEX_SEILER"])
@pytest.mark.parametrize("fmt,levels", [("AUTO", 0.0), ("UNORM16", 65535.0), ("UNORM8", 255.0)])
@pytest.mark.parametrize("nu,nv,nw", [(16, 16, 16), (32, 5, 8), (1, 1, 4), (7, 33, 12)])
def test_texture_tricubic_volume(variant, fmt, levels, nu, nv, nw):
    # Tricubic scalar volumes through the surface tiles one axis up: tile
    # (p, j) holds the u cubics C[.][j][l] in channel l, one filtered read per
    # (row u, j) gives Y[u][j][.], and the v and w stages are FP32 convex
    # combinations.  So the error is that of one filtered read of a tile
    # (axes x WERR of the largest channel range, plus half a code of it for
    # unorm texels), the same bound as the surfaces.
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(7300 + nu + 3 * nv + 7 * nw + int(levels))
    ctrl = rng.normal(size=(129, 4, 4, 4, 1)).astype(np.float32)
    ctrl[3] = -1.5                                                        # constant volume
    got = bez.bez_eval_volume(torch.from_numpy(ctrl).cuda(), nu, nv, nw, variant=bez.Variant[variant],
                              tex_format=bez.TexFormat[fmt]).cpu().numpy().astype(np.float64)
    ref = oracle.volume(ctrl, nu, nv, nw)
    b = ctrl[..., 0].astype(np.float64)                                  # [n][i][j][l]
    if variant == "TEX_DECASTELJAU":
        tile, axes = b, 3
    else:
        d1 = 3 * (b[:, 1] - b[:, 0]) - (b[:, 3] - b[:, 0])
        d2 = 3 * (b[:, 2] - b[:, 3]) - (b[:, 0] - b[:, 3])
        tile, axes = np.stack([b[:, 0], b[:, 3], b[:, 0] + d1, b[:, 3] + d2], 1), 2
    rng_jl = (tile.max(axis=1) - tile.min(axis=1)).max(axis=(1, 2))     # [n]
    mag = np.abs(tile).max(axis=(1, 2, 3))
    q = 0.5 / levels if levels else 0.0
    tol = (axes * WERR + q) * rng_jl + 12 * U * mag
    err = np.abs(got - ref).max(axis=(1, 2, 3, 4))
    assert np.all(err <= tol), (err / np.maximum(tol, 1e-30)).max()
    assert np.abs(got[3] + 1.5).max() <= 12 * U * 1.5                     # flat: exact up to the FP32 v, w stages
    if fmt == "AUTO":
        # texel centres: u = 0 and u = 1 read the corner texels exactly, and the
        # v, w stages at their ends select a single control point
        np.testing.assert_array_equal(got[:, 0, 0, 0, 0], ctrl[:, 0, 0, 0, 0])
        if nu > 1 and nv > 1 and nw > 1:
            np.testing.assert_array_equal(got[:, -1, -1, -1, 0], ctrl[:, -1, -1, -1, 0])


def test_texture_surface_unorm_from_half_storage():
    # FP16 control points with unorm16 tiles: the rescale works on the stored
    # half values, so the bound is the float-tile bound of those values
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(7200)
    c = torch.from_numpy(rng.uniform(-1, 1, (97, 4, 4, 3)).astype(np.float32)).cuda().half()
    got = bez.bez_eval_surface(c, 16, 24, variant=bez.Variant.TEX_SEILER,
                               tex_format=bez.TexFormat.UNORM16).cpu().numpy().astype(np.float64)
    b = c.float().cpu().numpy().astype(np.float64)
    ref = oracle.surface(b, 16, 24)
    d1 = 3 * (b[:, 1] - b[:, 0]) - (b[:, 3] - b[:, 0])
    d2 = 3 * (b[:, 2] - b[:, 3]) - (b[:, 0] - b[:, 3])
    tile = np.stack([b[:, 0], b[:, 3], b[:, 0] + d1, b[:, 3] + d2], 1)
    col_range = (tile.max(axis=1) - tile.min(axis=1)).max(axis=1)
    tol = (2 * WERR + 0.5 / 65535) * col_range + 8 * U * np.abs(tile).max(axis=(1, 2))
    assert np.all(np.abs(got - ref) <= tol[:, None, None, :])


def test_texture_surface_unsupported():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    tex = bez.Variant.TEX_DECASTELJAU
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval_surface(torch.zeros((2, 3, 4, 3), device="cuda"), 8, 8, variant=tex)   # not bicubic
    assert e.value.status == bez.Status.UNSUPPORTED
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval_surface(torch.zeros((2, 4, 4, 3), device="cuda"), 65, 8, variant=tex)  # rows > 64
    assert e.value.status == bez.Status.UNSUPPORTED
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval_surface(torch.zeros((2, 4, 4, 3), device="cuda", dtype=torch.bfloat16), 8, 8, variant=tex)
    assert e.value.status == bez.Status.UNSUPPORTED
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval_volume(torch.zeros((2, 4, 4, 4, 3), device="cuda"), 4, 4, 4, variant=tex)   # not scalar
    assert e.value.status == bez.Status.UNSUPPORTED
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval_volume(torch.zeros((2, 4, 4, 4, 1), device="cuda"), 4, 4, 6, variant=tex)   # nw % 4
    assert e.value.status == bez.Status.UNSUPPORTED
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval_volume(torch.zeros((2, 4, 4, 4, 1), device="cuda"), 33, 4, 4, variant=tex)  # rows > 32
    assert e.value.status == bez.Status.UNSUPPORTED
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval_volume(torch.zeros((2, 3, 4, 4, 1), device="cuda"), 4, 4, 4, variant=tex)   # not tricubic
    assert e.value.status == bez.Status.UNSUPPORTED


@pytest.mark.parametrize("share", [1, 2, 3, 5, 7])
@pytest.mark.parametrize("n_t", [1024, 77])
def test_coissue_length_mixes_texture_and_register_points(share, n_t):
    # In every 8 consecutive samples the first `share` come from the tex2D
    # Seiler tile and the rest from centred Horner; both use the bez_eval
    # draw and the same tile as TEX_SEILER, so the kernel's length must be
    # the polyline through TEX_SEILER points at j mod 8 < share and
    # HORNER_CENTRED points elsewhere, up to FP32 accumulation.
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(90 + share)
    n = 333
    ctrl = rng.uniform(-1, 1, size=(n, 4, 3)).astype(np.float32)
    kw = dict(n_t=n_t, t_mode="HASH", seed=5, stream_id=3)
    got = _run(torch, ctrl, variant="COISSUE", out_mode="POLYLINE_LENGTH", **kw, tex_share=share)
    p_tex = _run(torch, ctrl, variant="TEX_SEILER", **kw)[..., :3].astype(np.float64)
    p_reg = _run(torch, ctrl, variant="HORNER_CENTRED", **kw).astype(np.float64)
    use_tex = (np.arange(n_t) % 8) < share
    mixed = np.where(use_tex[None, :, None], p_tex, p_reg)
    L = oracle.polyline_length(mixed)
    assert np.all(np.abs(got - L) <= (n_t / 32 + 12) * U * L + 1e-7)


def test_coissue_default_share_and_unsupported():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(91)
    ctrl = rng.uniform(-1, 1, size=(40, 4, 3)).astype(np.float32)
    kw = dict(n_t=256, variant="COISSUE", out_mode="POLYLINE_LENGTH", t_mode="HASH", seed=1)
    np.testing.assert_array_equal(_run(torch, ctrl, **kw), _run(torch, ctrl, **kw, tex_share=2))
    c = torch.from_numpy(ctrl).cuda()
    co = dict(variant=bez.Variant.COISSUE, t_mode=bez.TMode.HASH)
    for args, status in [
        (dict(ctrl=c, n_t=64, out_mode=bez.OutMode.POINTS), bez.Status.UNSUPPORTED),
        (dict(ctrl=c[:, :3].contiguous(), n_t=64, out_mode=bez.OutMode.POLYLINE_LENGTH), bez.Status.UNSUPPORTED),
        (dict(ctrl=c, n_t=65537, out_mode=bez.OutMode.POLYLINE_LENGTH), bez.Status.UNSUPPORTED),
        (dict(ctrl=c, n_t=64, out_mode=bez.OutMode.POLYLINE_LENGTH, tex_share=8), bez.Status.INVALID_ARG),
    ]:
        with pytest.raises(bez.BezError) as e:
            bez.bez_eval(args.pop("ctrl"), None, **co, **args)
        assert e.value.status == status


@pytest.mark.parametrize("fmt,levels", [("UNORM16", 65535.0), ("UNORM8", 255.0)])
@pytest.mark.parametrize("variant,d", [("TEX_DECASTELJAU", 3), ("TEX_DECASTELJAU", 5), ("TEX_HYBRID", 3),
                                       ("TEX_HYBRID", 4), ("TEX_SEILER", 3), ("TEX_SEILER", 5), ("TEX_SEILER", 7)])
def test_texture_unorm_formats(fmt, levels, variant, d):
    # Sec. 2.3: unorm texels hold [0, 1]; each tile is stored as
    # (texel - lo) / scale with its own minimum and range and mapped back
    # after filtering, so the bound gains half a code of the tile's range
    # (filtering and the register lerps after it are convex).
    torch = need_gpu()
    rng = np.random.default_rng(80 + d)
    ctrl = rng.uniform(-1, 1, size=(777, d + 1, 3)).astype(np.float32)
    t = rng.uniform(0, 1, 53).astype(np.float32)
    got = _run(torch, ctrl, t, variant=variant, tex_format=fmt)
    ref = oracle.bezier(ctrl, t)
    err = np.linalg.norm(got - ref, axis=-1).max(axis=1)
    bound = texture_bound(variant, ctrl, texel_q=0.5 / levels) + 8 * U * np.abs(ctrl).max(axis=(1, 2))
    assert np.all(err <= bound), (err / bound).max()
    print(f"\n{variant} d={d} {fmt}: max normalised error {normalised_error(got, ref).max():.3g}")


def test_texture_unorm_length_and_unsupported():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(81)
    ctrl = rng.uniform(-1, 1, size=(64, 4, 3)).astype(np.float32)
    # the length path applies the same rescale: close to the float-texel length
    kw = dict(n_t=512, variant="TEX_SEILER", out_mode="POLYLINE_LENGTH", t_mode="HASH", seed=3)
    l32 = _run(torch, ctrl, **kw)
    l16 = _run(torch, ctrl, **kw, tex_format="UNORM16")
    assert np.all(np.abs(l16 - l32) <= 2e-3 * l32)
    c = torch.from_numpy(ctrl).cuda()
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval_piecewise(torch.zeros((2, 9, 3), device="cuda"), 4, 2, n_t=8, t_mode=bez.TMode.UNIFORM,
                               variant=bez.Variant.TEX_DECASTELJAU, tex_format=bez.TexFormat.UNORM8)
    assert e.value.status == bez.Status.UNSUPPORTED
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval(c, None, n_t=8, t_mode=bez.TMode.UNIFORM, variant=bez.Variant.TEX_SEILER, tex_format=7)
    assert e.value.status == bez.Status.INVALID_ARG

