"""GPU parity of the register curve evaluators (bez_eval) against the FP64
oracle, through the C ABI.

Bar (FP32 arithmetic): per-curve max normalised error <= 1e-6 for the
centred-Horner, Bernstein, de Casteljau and Seiler forms at degrees 1..7.
The raw power-basis Horner baseline is checked against its a-priori FP32
error bound instead (it is known to miss 1e-6 from degree 3).  Degrees 8..15
run the runtime-degree kernels and are held to 64 d u max|b| (a logic error
shows up at the size of the control points).  Exactness properties
(endpoints, partition of unity, dyadic inputs) are checked bit for bit."""
import numpy as np
import pytest

import oracle
from gpu_util import horner_bound, need_gpu, normalised_error, normalised_error_ctrl

pytestmark = pytest.mark.gpu

FP32_BAR = 1e-6
ACCURATE = ["HORNER_CENTRED", "BERNSTEIN", "DECASTELJAU", "SEILER"]
ALL = ["HORNER"] + ACCURATE


def _run(torch, ctrl, t=None, n_t=None, variant="SEILER", out_mode="POINTS", t_mode=None, seed=0, stream_id=0,
         dtype=None):
    from paper_2603_15447_gb300 import bez
    c = torch.from_numpy(ctrl).cuda()
    if dtype is not None:
        c = c.to(dtype)
    tt = None if t is None else torch.from_numpy(np.ascontiguousarray(t, np.float32)).cuda()
    out = bez.bez_eval(c, tt, n_t=n_t, variant=bez.Variant[variant], out_mode=bez.OutMode[out_mode],
                       t_mode=None if t_mode is None else bez.TMode[t_mode], seed=seed, stream_id=stream_id)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _ctrl(rng, B, d, dim):
    return rng.uniform(-1, 1, size=(B, d + 1, dim)).astype(np.float32)


@pytest.mark.parametrize("variant", ALL)
@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6, 7])
def test_points_shared_t(variant, d):
    torch = need_gpu()
    rng = np.random.default_rng(100 + d)
    ctrl = _ctrl(rng, 1003, d, 3)                 # ragged: not a multiple of the 8-curve block
    t = rng.uniform(0, 1, 77).astype(np.float32)  # ragged: not a multiple of the 32-lane tile
    got = _run(torch, ctrl, t, variant=variant)
    ref = oracle.bezier(ctrl, t)
    if variant == "HORNER":
        assert np.all(np.abs(got - ref) <= horner_bound(ctrl.astype(np.float64), t.astype(np.float64)))
    else:
        assert normalised_error(got, ref).max() <= FP32_BAR


@pytest.mark.parametrize("variant", ALL)
@pytest.mark.parametrize("dim", [1, 2, 4])
def test_points_other_dims_per_curve_t(variant, dim):
    torch = need_gpu()
    rng = np.random.default_rng(200 + dim)
    d = 3
    ctrl = _ctrl(rng, 517, d, dim)
    t = rng.uniform(0, 1, (517, 45)).astype(np.float32)
    got = _run(torch, ctrl, t, variant=variant, t_mode="PER_CURVE")
    ref = oracle.bezier(ctrl, t)
    if variant == "HORNER":
        assert np.all(np.abs(got - ref) <= horner_bound(ctrl.astype(np.float64), t.astype(np.float64)))
    else:
        assert normalised_error_ctrl(got, ref, ctrl).max() <= FP32_BAR


@pytest.mark.parametrize("variant", ALL)
@pytest.mark.parametrize("d", [8, 11, 15])
def test_points_high_degree_runtime_kernels(variant, d):
    torch = need_gpu()
    rng = np.random.default_rng(300 + d)
    ctrl = _ctrl(rng, 129, d, 3)
    t = rng.uniform(0, 1, 50).astype(np.float32)
    got = _run(torch, ctrl, t, variant=variant)
    ref = oracle.bezier(ctrl, t)
    if variant == "HORNER":
        assert np.all(np.abs(got - ref) <= horner_bound(ctrl.astype(np.float64), t.astype(np.float64)))
    else:
        M = np.abs(ctrl).max(axis=(1, 2))[:, None, None]
        assert np.all(np.abs(got - ref) <= 64 * d * 2.0 ** -24 * M)


@pytest.mark.parametrize("variant", ALL)
def test_uniform_grid_and_hash_modes(variant):
    torch = need_gpu()
    rng = np.random.default_rng(400)
    ctrl = _ctrl(rng, 300, 3, 3)
    got = _run(torch, ctrl, n_t=256, variant=variant, t_mode="UNIFORM")
    ref = oracle.bezier_grid(ctrl, 256)
    tol_ok = (lambda g, r, tt: np.all(np.abs(g - r) <= horner_bound(ctrl.astype(np.float64), tt))) \
        if variant == "HORNER" else (lambda g, r, tt: normalised_error(g, r).max() <= FP32_BAR)
    assert tol_ok(got, ref, oracle.grid(256))
    got = _run(torch, ctrl, n_t=100, variant=variant, t_mode="HASH", seed=77, stream_id=5)
    th = oracle.hash_t(77, 5, 0, 300, 100)
    assert tol_ok(got, oracle.bezier(ctrl, th), th)


@pytest.mark.parametrize("variant", ACCURATE)
def test_exact_endpoints_partition_clamp_nan(variant):
    torch = need_gpu()
    rng = np.random.default_rng(500)
    for d in (1, 2, 3, 5, 7, 9):
        ctrl = _ctrl(rng, 64, d, 3)
        t = np.array([0.0, 1.0, -3.0, 7.0, np.nan], np.float32)
        got = _run(torch, ctrl, t, variant=variant)
        if variant != "HORNER_CENTRED":
            np.testing.assert_array_equal(got[:, 0], ctrl[:, 0])
            np.testing.assert_array_equal(got[:, 1], ctrl[:, d])
        np.testing.assert_array_equal(got[:, 2], got[:, 0])
        np.testing.assert_array_equal(got[:, 3], got[:, 1])
        assert np.isnan(got[:, 4]).all()
        if variant in ("DECASTELJAU", "SEILER"):
            const = np.repeat(ctrl[:, :1], d + 1, axis=1)
            tt = rng.uniform(0, 1, 64).astype(np.float32)
            np.testing.assert_array_equal(_run(torch, const, tt, variant=variant),
                                          np.repeat(const[:, :1], 64, axis=1))


@pytest.mark.parametrize("variant", ["DECASTELJAU", "SEILER", "BERNSTEIN", "HORNER_CENTRED"])
def test_bitexact_small_integers_dyadic_t(variant):
    # Control points in [-8, 8] and t = k/32: every FP32 intermediate of the
    # cubic forms stays exact (at most 4 + 3*5 + 4 bits), so the GPU result
    # must equal the oracle (itself exact here) bit for bit.
    torch = need_gpu()
    rng = np.random.default_rng(600)
    ctrl = rng.integers(-8, 9, size=(256, 4, 3)).astype(np.float32)
    t = (np.arange(33) / 32).astype(np.float32)
    got = _run(torch, ctrl, t, variant=variant)
    np.testing.assert_array_equal(got, oracle.bezier(ctrl, t).astype(np.float32))


def test_half_and_bfloat16_storage():
    torch = need_gpu()
    rng = np.random.default_rng(700)
    ctrl = _ctrl(rng, 500, 3, 3)
    t = rng.uniform(0, 1, 64).astype(np.float32)
    for dt, name in ((torch.float16, "f16"), (torch.bfloat16, "bf16")):
        stored = torch.from_numpy(ctrl).to(dt).float().numpy()      # the values the kernel reads
        got = _run(torch, ctrl, t, variant="SEILER", dtype=dt)
        assert normalised_error(got, oracle.bezier(stored, t)).max() <= FP32_BAR, name


# A lane sums a run of consecutive segment lengths, then lanes combine by a
# butterfly.  The centred-Horner length kernels give a lane runs of n_t/16
# (two curves per warp), n_t/8 (four, from 128 samples) or n_t/4 (eight, from
# 256), and the other kernels n_t/32, so n_t/4 bounds the run term of every
# form.
def _length_tol(ref_pts, L_ref, n_t):
    diag = np.maximum(np.linalg.norm(ref_pts.max(axis=1) - ref_pts.min(axis=1), axis=-1), 2.0 ** -4)
    u = 2.0 ** -24
    return 2 * (n_t - 1) * FP32_BAR * diag + (6 + n_t / 4 + 6) * u * L_ref + 1e-7


@pytest.mark.parametrize("variant", ALL)
def test_polyline_length_hash(variant):
    torch = need_gpu()
    rng = np.random.default_rng(800)
    n, n_t = 777, 1024
    ctrl = _ctrl(rng, n, 3, 3)
    got = _run(torch, ctrl, n_t=n_t, variant=variant, out_mode="POLYLINE_LENGTH", t_mode="HASH", seed=20260316,
               stream_id=2)
    th = oracle.hash_t(20260316, 2, 0, n, n_t)
    pts = oracle.bezier(ctrl, th)
    L = oracle.polyline_length(pts)
    if variant == "HORNER":
        # Horner's point error bound replaces the 1e-6 bar in the tolerance
        e = np.linalg.norm(horner_bound(ctrl.astype(np.float64), th), axis=-1).max(axis=1)
        tol = 2 * (n_t - 1) * e + 20 * 2.0 ** -24 * L * (n_t / 32 + 12)
    else:
        tol = _length_tol(pts, L, n_t)
    assert np.all(np.abs(got - L) <= tol)


@pytest.mark.parametrize("n_t", [3, 5, 127, 65536, 65537])
def test_polyline_length_hash_index_width(n_t):
    # up to 2^16 samples the draw uses the pre-mixed curve key and runs of a
    # multiple of 4 samples per lane; above that the plain key; both give the
    # oracle's draw
    torch = need_gpu()
    rng = np.random.default_rng(4000 + n_t)
    n = 5
    ctrl = _ctrl(rng, n, 3, 3)
    got = _run(torch, ctrl, n_t=n_t, variant="HORNER_CENTRED", out_mode="POLYLINE_LENGTH", t_mode="HASH",
               seed=99, stream_id=7)
    th = oracle.hash_t(99, 7, 0, n, n_t)
    pts = oracle.bezier(ctrl, th)
    L = oracle.polyline_length(pts)
    assert np.all(np.abs(got - L) <= _length_tol(pts, L, n_t))


@pytest.mark.parametrize("n_t", [0, 1, 2, 31, 33, 100])
def test_polyline_length_edge_sizes(n_t):
    torch = need_gpu()
    rng = np.random.default_rng(900 + n_t)
    ctrl = _ctrl(rng, 41, 3, 3)
    t = np.sort(rng.uniform(0, 1, (41, n_t)).astype(np.float32), axis=1)
    got = _run(torch, ctrl, t, variant="DECASTELJAU", out_mode="POLYLINE_LENGTH", t_mode="PER_CURVE")
    if n_t == 0:
        np.testing.assert_array_equal(got, 0.0)
        return
    pts = oracle.bezier(ctrl, t)
    L = oracle.polyline_length(pts)
    assert np.all(np.abs(got - L) <= _length_tol(pts, L, n_t))


def test_empty_inputs_and_invalid_args():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    empty = _run(torch, np.zeros((0, 4, 3), np.float32), np.zeros(5, np.float32))
    assert empty.shape == (0, 5, 3)
    ctrl = torch.zeros((4, 4, 3), device="cuda")
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval(ctrl.reshape(4, 4, 3)[:, :, :0], torch.zeros(3, device="cuda"))
    assert e.value.status == bez.Status.INVALID_ARG
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval(torch.zeros((4, 17, 3), device="cuda"), torch.zeros(3, device="cuda"))
    assert e.value.status == bez.Status.UNSUPPORTED
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval(ctrl, None, n_t=3, t_mode=bez.TMode.SHARED)
    assert e.value.status == bez.Status.INVALID_ARG


def test_host_buffers_are_staged():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(1000)
    ctrl = _ctrl(rng, 200, 3, 3)
    t = rng.uniform(0, 1, 40).astype(np.float32)
    got_np = bez.bez_eval(ctrl, t, variant=bez.Variant.SEILER)                       # NumPy host arrays
    got_pinned = bez.bez_eval(torch.from_numpy(ctrl).pin_memory(), torch.from_numpy(t).pin_memory(),
                              variant=bez.Variant.SEILER)                            # pinned torch tensors
    dev = _run(torch, ctrl, t, variant="SEILER")
    np.testing.assert_array_equal(got_np, dev)
    np.testing.assert_array_equal(got_pinned.numpy(), dev)


def test_launch_accounting_and_timing():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    ctx = bez.context(0)
    ctx.reset_stats()
    ctx.set_timing(True)
    c = torch.rand((64, 4, 3), device="cuda")
    for _ in range(3):
        bez.bez_eval(c, None, n_t=128, t_mode=bez.TMode.UNIFORM)
    s = ctx.stats()
    ctx.set_timing(False)
    assert s["launches"] == 3 and s["timed_launches"] == 3 and s["timed_ms"] > 0


def _centred_coeffs(ctrl):
    """Power coefficients about t = 1/2 of each Bezier curve, FP64 [B][d+1][dim]."""
    from math import comb
    from numpy.polynomial import polynomial as Pn
    B, d1, dim = ctrl.shape
    d = d1 - 1
    out = np.zeros((B, d1, dim))
    shift = np.array([0.5, 1.0])  # t = u + 1/2
    for c in range(B):
        for k in range(dim):
            poly = np.zeros(d1)
            for i in range(d1):
                basis = comb(d, i) * Pn.polymul(Pn.polypow([1.0, -1.0], d - i), Pn.polypow([0.0, 1.0], i))
                poly = Pn.polyadd(poly, float(ctrl[c, i, k]) * basis)[:d1]
            comp = np.zeros(1)
            for i in reversed(range(d1)):          # Horner composition poly(u + 1/2)
                comp = Pn.polyadd(Pn.polymul(comp, shift), [poly[i]])
            out[c, :, k] = np.pad(comp, (0, d1 - len(comp)))[:d1]
    return out


@pytest.mark.parametrize("d", [1, 3, 5, 7])
@pytest.mark.parametrize("t_mode", ["SHARED", "HASH"])
def test_half2_arithmetic_points(d, t_mode):
    # Centred Horner in half2: coefficients rounded to half (2^-11), u = t - 1/2
    # rounded to half (2^-13 absolute, times |C'|), and 2d half FMAs, each
    # rounding by 2^-11 of a partial sum bounded by S = sum_i |c_i| |u|^i.
    torch = need_gpu()
    rng = np.random.default_rng(300 + d)
    n = 257
    ctrl = _ctrl(rng, n, d, 3)
    if t_mode == "SHARED":
        t = rng.uniform(0, 1, 131).astype(np.float32)
        got = _run(torch, ctrl, t, variant="HALF2")
        tt = np.broadcast_to(t, (n, t.size))
    else:
        got = _run(torch, ctrl, n_t=131, variant="HALF2", t_mode="HASH", seed=4, stream_id=1)
        tt = oracle.hash_t(4, 1, 0, n, 131)
    ref = oracle.bezier(ctrl, tt if t_mode == "HASH" else t)
    c = _centred_coeffs(ctrl.astype(np.float64))                       # [n][d+1][3]
    u = np.abs(tt.astype(np.float64) - 0.5)                            # [n][n_t]
    S = np.einsum("nik,nti->ntk", np.abs(c), u[..., None] ** np.arange(d + 1))
    dmax = np.abs(np.diff(ctrl.astype(np.float64), axis=1)).max(axis=1)   # [n][3]
    tol = (2 * d + 4) * 2.0 ** -11 * S + 2.0 ** -12 * d * dmax[:, None, :] + 1e-6
    assert np.all(np.abs(got - ref) <= tol)
    print(f"\nHALF2 d={d} {t_mode}: max normalised error {normalised_error(got, ref).max():.3g}")


@pytest.mark.parametrize("n_t", [1024, 77, 1])
def test_half2_length_is_polyline_of_its_points(n_t):
    torch = need_gpu()
    rng = np.random.default_rng(310)
    ctrl = _ctrl(rng, 129, 3, 3)
    kw = dict(n_t=n_t, variant="HALF2", t_mode="HASH", seed=8, stream_id=2)
    L = _run(torch, ctrl, out_mode="POLYLINE_LENGTH", **kw)
    pts = _run(torch, ctrl, **kw).astype(np.float64)
    want = oracle.polyline_length(pts)
    assert np.all(np.abs(L - want) <= (n_t / 32 + 12) * 2.0 ** -24 * want + 1e-7)


def test_half2_unsupported():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    for shape in [(4, 4, 2), (4, 9, 3)]:
        with pytest.raises(bez.BezError) as e:
            bez.bez_eval(torch.zeros(shape, device="cuda"), torch.zeros(3, device="cuda"), variant=bez.Variant.HALF2)
        assert e.value.status == bez.Status.UNSUPPORTED


@pytest.mark.parametrize("out_mode,t_mode,pinned", [("POLYLINE_LENGTH", "HASH", True), ("POINTS", "HASH", False),
                                                    ("POLYLINE_LENGTH", "SHARED", False), ("POINTS", "UNIFORM", True)])
def test_pipelined_host_call_matches_device_call(out_mode, t_mode, pinned):
    # Host control points and host output: the call runs as chunks whose
    # copies overlap the evaluation of neighbouring chunks; every chunk hashes
    # its curves by their global index, so the result equals the device call.
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    rng = np.random.default_rng(500)
    n = 70001
    n_t = 33 if out_mode == "POINTS" else 256
    ctrl = _ctrl(rng, n, 3, 3)
    t = rng.uniform(0, 1, n_t).astype(np.float32) if t_mode == "SHARED" else None
    kw = dict(n_t=None if t is not None else n_t, variant=bez.Variant.HORNER_CENTRED, out_mode=bez.OutMode[out_mode],
              t_mode=bez.TMode[t_mode], seed=12, stream_id=3)
    dev = bez.bez_eval(torch.from_numpy(ctrl).cuda(), None if t is None else torch.from_numpy(t).cuda(), **kw)
    host_ctrl = torch.from_numpy(ctrl)
    if pinned:
        host_ctrl = host_ctrl.pin_memory()
    host = bez.bez_eval(host_ctrl, None if t is None else torch.from_numpy(t), **kw)
    assert host.device.type == "cpu"
    np.testing.assert_array_equal(host.numpy(), dev.cpu().numpy())


def _ctrl_diag(ctrl):
    c = ctrl.astype(np.float64)
    return np.linalg.norm(c.max(axis=1) - c.min(axis=1), axis=-1)


def test_headline_length_kernel_at_full_size():
    # The fused draw + centred Horner + length kernel in the launch shape the
    # benchmark times: 1,048,575 cubic 3D curves (the warps' last unit of
    # curves partial) x 1024 hashed parameters, so the grid is not persistent
    # and every warp walks several units with the next unit's control points
    # prefetched.  Every curve's length is compared with
    # the oracle's; the tolerance takes the 1e-6 point bar over the control
    # polygon's diagonal (>= the curve's), and a sample spread over the batch
    # is held to the curve-diagonal tolerance of the smaller tests.
    torch = need_gpu()
    from paper_2603_15447_gb300 import synth
    seed = synth.BASE_SEED + 1
    n, n_t = (1 << 20) - 1, 1024
    ctrl = synth.precision(seed=seed, n_curves=n)
    got = _run(torch, ctrl, n_t=n_t, variant="HORNER_CENTRED", out_mode="POLYLINE_LENGTH", t_mode="HASH",
               seed=seed, stream_id=synth.PRECISION_T_STREAM)
    chunk = 1 << 15
    L = np.concatenate([oracle.hashed_bezier_polyline_length(ctrl[s:s + chunk], n_t, seed,
                                                             synth.PRECISION_T_STREAM, c0=s)
                        for s in range(0, n, chunk)])
    u = 2.0 ** -24
    tol = 2 * (n_t - 1) * FP32_BAR * _ctrl_diag(ctrl) + (6 + n_t / 4 + 6) * u * L + 1e-7
    assert np.all(np.abs(got - L) <= tol), (np.abs(got - L) / tol).max()
    idx = np.unique(np.concatenate([np.arange(0, n, 97), [n - 2, n - 1]]))
    th = np.concatenate([oracle.hash_t(seed, synth.PRECISION_T_STREAM, int(c), 1, n_t) for c in idx])
    pts = oracle.bezier(ctrl[idx], th)
    assert np.all(np.abs(got[idx] - L[idx]) <= _length_tol(pts, L[idx], n_t))
    print(f"\nfull-size headline: max relative length error {np.max(np.abs(got - L) / L):.3g}")


@pytest.mark.parametrize("n_t,degree", [(128, 3), (200, 4), (96, 1), (256, 2), (333, 4), (512, 3), (700, 1),
                                         (2051, 4)])
def test_fused_length_kernels_block_scheduled(n_t, degree):
    # The centred-Horner length kernels by samples per curve: two curves per
    # warp below 128, four from 128, eight from 256.  300,001 curves: more
    # units than resident warps, so every warp walks several with the next
    # one's control points prefetched, and the last unit is partial.  Every
    # length is compared with the oracle.
    torch = need_gpu()
    rng = np.random.default_rng(7100 + n_t)
    n = 300_001 if n_t < 1000 else 60_001
    ctrl = _ctrl(rng, n, degree, 3)
    seed, stream = 4242, 3
    got = _run(torch, ctrl, n_t=n_t, variant="HORNER_CENTRED", out_mode="POLYLINE_LENGTH", t_mode="HASH",
               seed=seed, stream_id=stream)
    chunk = 1 << 15
    L = np.concatenate([oracle.hashed_bezier_polyline_length(ctrl[s:s + chunk], n_t, seed, stream, c0=s)
                        for s in range(0, n, chunk)])
    u = 2.0 ** -24
    tol = 2 * (n_t - 1) * FP32_BAR * _ctrl_diag(ctrl) + (6 + n_t / 4 + 6) * u * L + 1e-7
    assert np.all(np.abs(got - L) <= tol), (np.abs(got - L) / tol).max()


@pytest.mark.parametrize("variant", ["HORNER_CENTRED", "DECASTELJAU"])
def test_points_kernel_at_block_scheduled_size(variant):
    # k_curve (points) with more curves than resident warps: 50,001 curves
    # (ragged against the 8-curve warp blocks) x 256 hashed parameters
    torch = need_gpu()
    rng = np.random.default_rng(1234)
    n, n_t = 50001, 256
    ctrl = _ctrl(rng, n, 3, 3)
    got = _run(torch, ctrl, n_t=n_t, variant=variant, t_mode="HASH", seed=77, stream_id=5)
    th = oracle.hash_t(77, 5, 0, n, n_t)
    ref = oracle.bezier(ctrl, th)
    assert normalised_error(got, ref).max() <= FP32_BAR
