"""GPU parity of C0 piecewise chains (bez_eval_piecewise, paper Sec. 2.1).

Register evaluators are held to the FP32 bar (1e-6 of the chain's bounding
box diagonal).  The zig-zag texture is held to the texture tolerance model
of test_tex_gpu: two filtered axes, each moving the point by at most
(weight error) x (texel range of the 2x2 window read).  The texels are rebuilt here
from the paper's construction (end points in alternating rows, free texels
F_k + F_(k+1) = 2 P_(2k+1)) with the documented choice of F_0."""
import numpy as np
import pytest

import oracle
from gpu_util import need_gpu, normalised_error, normalised_error_ctrl

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
WERR = 2.0 ** -8 + 2.0 ** -11
FP32_BAR = 1e-6


def _run(torch, ctrl, n_seg, degree, t=None, n_t=None, variant="DECASTELJAU", out_mode="POINTS", t_mode=None,
         seed=0, stream_id=0, half=False):
    from paper_2603_15447_gb300 import bez
    c = torch.from_numpy(ctrl).cuda()
    if half:
        c = c.half()
    tt = None if t is None else torch.from_numpy(np.ascontiguousarray(t, np.float32)).cuda()
    out = bez.bez_eval_piecewise(c, n_seg, degree, tt, n_t=n_t, variant=bez.Variant[variant],
                                 out_mode=bez.OutMode[out_mode],
                                 t_mode=None if t_mode is None else bez.TMode[t_mode], seed=seed,
                                 stream_id=stream_id)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def zigzag_texels(P):
    """[N+1] columns x 2 rows texture (rows, cols, dim) of one chain, with
    F_0 minimising max |F_k| per component."""
    P = P.astype(np.float64)
    N = (P.shape[0] - 1) // 2
    G = np.zeros((N + 1, P.shape[1]))
    for s in range(N):
        G[s + 1] = 2 * P[2 * s + 1] - G[s]
    H = G * np.array([(-1) ** k for k in range(N + 1)])[:, None]
    F0 = -(H.max(axis=0) + H.min(axis=0)) / 2
    T = np.zeros((2, N + 1, P.shape[1]))
    F = F0
    for k in range(N + 1):
        T[k % 2, k] = P[2 * k]
        T[1 - k % 2, k] = F
        if k < N:
            F = 2 * P[2 * k + 1] - F
    return T


def zigzag_bound(ctrl, texel_eps=U):
    """Two filtered axes x (2^-8 + 2^-11) x the texel range of the 2x2
    window read for a segment, maximised over the chain's windows (the
    tolerance model of test_tex_gpu), plus texel rounding."""
    out = np.empty(ctrl.shape[0])
    for c in range(ctrl.shape[0]):
        T = zigzag_texels(ctrl[c])                       # [2][N+1][dim]
        win = np.concatenate([T[:, :-1], T[:, 1:]], axis=0)   # [4][N][dim] windows
        rng_w = np.linalg.norm(win.max(axis=0) - win.min(axis=0), axis=-1).max()
        mag = np.abs(T).max()
        out[c] = 2 * WERR * rng_w + (8 * texel_eps + 12 * U) * mag * np.sqrt(ctrl.shape[2])
    return out


@pytest.mark.parametrize("variant", ["HORNER_CENTRED", "BERNSTEIN", "DECASTELJAU", "SEILER"])
@pytest.mark.parametrize("degree,dim", [(2, 3), (3, 3), (1, 3), (5, 3), (2, 1), (3, 4)])
def test_register_chains(variant, degree, dim):
    torch = need_gpu()
    rng = np.random.default_rng(10 * degree + dim)
    n_seg = 9
    ctrl = rng.uniform(-1, 1, size=(203, n_seg * degree + 1, dim)).astype(np.float32)
    t = (rng.uniform(0, 1, (203, 61)) * n_seg).astype(np.float32)
    t[:, :3] = [0.0, n_seg, 4.0]                      # ends and an interior joint
    got = _run(torch, ctrl, n_seg, degree, t, variant=variant, t_mode="PER_CURVE")
    ref = oracle.chain(ctrl, n_seg, degree, t)
    err = normalised_error(got, ref) if dim == 3 else normalised_error_ctrl(got, ref, ctrl)
    assert err.max() <= FP32_BAR


def test_register_chain_horner_baseline_runs():
    torch = need_gpu()
    rng = np.random.default_rng(3)
    ctrl = rng.uniform(-1, 1, size=(50, 2 * 6 + 1, 3)).astype(np.float32)
    t = (rng.uniform(0, 1, 40) * 6).astype(np.float32)
    got = _run(torch, ctrl, 6, 2, t, variant="HORNER")
    ref = oracle.chain(ctrl, 6, 2, t)
    assert np.abs(got - ref).max() <= 64 * U * 4      # quadratic Horner, |a_k| <= 4


@pytest.mark.parametrize("n_seg", [1, 3, 64])
def test_zigzag_texture_points(n_seg):
    torch = need_gpu()
    rng = np.random.default_rng(20 + n_seg)
    ctrl = rng.uniform(-1, 1, size=(301, 2 * n_seg + 1, 3)).astype(np.float32)
    t = (rng.uniform(0, 1, 97) * n_seg).astype(np.float32)
    t[:2] = [0.0, n_seg]
    got = _run(torch, ctrl, n_seg, 2, t, variant="TEX_DECASTELJAU")
    ref = oracle.chain(ctrl, n_seg, 2, t)
    err = np.linalg.norm(got - ref, axis=-1).max(axis=1)
    bound = zigzag_bound(ctrl)
    assert np.all(err <= bound), (err / bound).max()
    # end points and joints are texel centres: exact
    np.testing.assert_array_equal(got[:, 0], ctrl[:, 0])
    np.testing.assert_array_equal(got[:, 1], ctrl[:, -1])
    print(f"\nzig-zag N={n_seg}: max normalised error {normalised_error(got, ref).max():.3g}, "
          f"error/bound {(err / bound).max():.3f}")


def test_zigzag_joints_exact_and_nan():
    torch = need_gpu()
    rng = np.random.default_rng(30)
    n_seg = 7
    ctrl = rng.uniform(-1, 1, size=(64, 2 * n_seg + 1, 3)).astype(np.float32)
    t = np.array(list(range(n_seg + 1)) + [-2.0, 99.0, np.nan], np.float32)
    got = _run(torch, ctrl, n_seg, 2, t, variant="TEX_DECASTELJAU")
    np.testing.assert_array_equal(got[:, :n_seg + 1], ctrl[:, ::2])
    np.testing.assert_array_equal(got[:, n_seg + 1], ctrl[:, 0])
    np.testing.assert_array_equal(got[:, n_seg + 2], ctrl[:, -1])
    assert np.isnan(got[:, -1]).all()


def test_zigzag_modes_dims_half():
    torch = need_gpu()
    rng = np.random.default_rng(40)
    n_seg = 16
    for dim in (1, 2, 4):
        ctrl = rng.uniform(-1, 1, size=(100, 2 * n_seg + 1, dim)).astype(np.float32)
        t = (rng.uniform(0, 1, (100, 50)) * n_seg).astype(np.float32)
        got = _run(torch, ctrl, n_seg, 2, t, variant="TEX_DECASTELJAU", t_mode="PER_CURVE")
        err = np.linalg.norm(got - oracle.chain(ctrl, n_seg, 2, t), axis=-1).max(axis=1)
        assert np.all(err <= zigzag_bound(ctrl))
    ctrl = rng.uniform(-1, 1, size=(100, 2 * n_seg + 1, 3)).astype(np.float32)
    got = _run(torch, ctrl, n_seg, 2, n_t=77, variant="TEX_DECASTELJAU", t_mode="UNIFORM")
    tu = (np.float32(n_seg) * (np.arange(77, dtype=np.float32) / np.float32(76))).astype(np.float32)
    err = np.linalg.norm(got - oracle.chain(ctrl, n_seg, 2, tu), axis=-1).max(axis=1)
    assert np.all(err <= zigzag_bound(ctrl))
    got = _run(torch, ctrl, n_seg, 2, n_t=64, variant="TEX_DECASTELJAU", t_mode="HASH", seed=5, stream_id=1)
    th = (np.float32(n_seg) * oracle.hash_t(5, 1, 0, 100, 64).astype(np.float32)).astype(np.float32)
    err = np.linalg.norm(got - oracle.chain(ctrl, n_seg, 2, th), axis=-1).max(axis=1)
    assert np.all(err <= zigzag_bound(ctrl))
    stored = ctrl.astype(np.float16).astype(np.float32)
    t = (rng.uniform(0, 1, 40) * n_seg).astype(np.float32)
    got = _run(torch, ctrl, n_seg, 2, t, variant="TEX_DECASTELJAU", half=True)
    err = np.linalg.norm(got - oracle.chain(stored, n_seg, 2, t), axis=-1).max(axis=1)
    assert np.all(err <= zigzag_bound(stored, texel_eps=2.0 ** -11))


@pytest.mark.parametrize("variant", ["DECASTELJAU", "HORNER_CENTRED", "TEX_DECASTELJAU"])
def test_chain_polyline_length_hash(variant):
    torch = need_gpu()
    rng = np.random.default_rng(50)
    n, n_seg, n_t = 64, 64, 4096
    ctrl = rng.uniform(-1, 1, size=(n, 2 * n_seg + 1, 3)).astype(np.float32)
    got = _run(torch, ctrl, n_seg, 2, n_t=n_t, variant=variant, out_mode="POLYLINE_LENGTH", t_mode="HASH",
               seed=20260316, stream_id=12)
    th = (np.float32(n_seg) * oracle.hash_t(20260316, 12, 0, n, n_t).astype(np.float32)).astype(np.float32)
    pts = oracle.chain(ctrl, n_seg, 2, th)
    L = oracle.polyline_length(pts)
    if variant != "TEX_DECASTELJAU":
        diag = np.maximum(np.linalg.norm(pts.max(axis=1) - pts.min(axis=1), axis=-1), 2.0 ** -4)
        e = FP32_BAR * diag
    else:
        e = zigzag_bound(ctrl)
    tol = 2 * (n_t - 1) * e + (n_t / 32 + 12) * U * L
    assert np.all(np.abs(got - L) <= tol)


def test_chain_argument_errors():
    torch = need_gpu()
    from paper_2603_15447_gb300 import bez
    ctrl = torch.zeros((2, 9, 3), device="cuda")
    with pytest.raises(bez.BezError) as e:                  # zig-zag textures: quadratic or cubic segments
        bez.bez_eval_piecewise(ctrl, 2, 4, torch.zeros(4, device="cuda"), variant=bez.Variant.TEX_DECASTELJAU)
    assert e.value.status == bez.Status.UNSUPPORTED
    with pytest.raises(bez.BezError) as e:                  # cubic zig-zag: no spread layout
        bez.bez_eval_piecewise(torch.zeros((2, 7, 3), device="cuda"), 2, 3, torch.zeros(4, device="cuda"),
                               variant=bez.Variant.TEX_DECASTELJAU, tex_spread=2)
    assert e.value.status == bez.Status.UNSUPPORTED
    with pytest.raises(bez.BezError) as e:                  # zig-zag texels: unorm8 is too coarse
        bez.bez_eval_piecewise(torch.zeros((2, 5, 3), device="cuda"), 2, 2, torch.zeros(4, device="cuda"),
                               variant=bez.Variant.TEX_DECASTELJAU, tex_format=bez.TexFormat.UNORM8)
    assert e.value.status == bez.Status.UNSUPPORTED
    with pytest.raises(bez.BezError) as e:                  # unorm16: quadratic chains only
        bez.bez_eval_piecewise(torch.zeros((2, 7, 3), device="cuda"), 2, 3, torch.zeros(4, device="cuda"),
                               variant=bez.Variant.TEX_DECASTELJAU, tex_format=bez.TexFormat.UNORM16)
    assert e.value.status == bez.Status.UNSUPPORTED
    with pytest.raises(bez.BezError) as e:
        bez.bez_eval_piecewise(torch.zeros((2, 1, 3), device="cuda"), 0, 2, torch.zeros(4, device="cuda"))
    assert e.value.status == bez.Status.INVALID_ARG
