"""Pins for the oracle's Bezier, chain and polyline functions (CPU only).

The oracle's Bernstein sum is checked against routes that do not share its
formula: exact rational de Casteljau (paper Sec. 2), the paper's Seiler
recursion and texture layouts in exact arithmetic (Sec. 3-4), exact linear
texture filtering of the zig-zag chain texture (Sec. 2.1, Eq. 1-2), SciPy's
Bernstein polynomial class, and invariants (endpoint interpolation,
partition of unity, degree elevation)."""
import json
import os
import random
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
from exact import (bernstein_exact, bilinear, decasteljau, decasteljau_texture, lerp, seiler_eval,
                   seiler_terms, seiler_texture, trilinear, zigzag_sample, zigzag_texture, zigzag3_sample,
                   zigzag3_texture)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_int_ctrl(rng, B, d, dim, lo=-8, hi=8):
    return np.array([[[rng.randint(lo, hi) for _ in range(dim)] for _ in range(d + 1)] for _ in range(B)],
                    dtype=np.float64)


@pytest.mark.parametrize("d,m", [(1, 20), (2, 14), (3, 12), (5, 7), (7, 5)])
def test_bernstein_bitexact_vs_rational_decasteljau(d, m):
    # Integer control points and dyadic t keep every FP64 intermediate exact
    # (d*m + 13 <= 53 bits), so the Bernstein sum must equal exact de Casteljau.
    rng = random.Random(1000 + d)
    B, dim = 6, 3
    ctrl = _rand_int_ctrl(rng, B, d, dim)
    ks = sorted(rng.sample(range(0, 2 ** m + 1), 16)) + [0, 2 ** m]
    t = np.array([k / 2 ** m for k in ks])
    got = oracle.bezier(ctrl, t)
    for c in range(B):
        for j, k in enumerate(ks):
            tf = F(k, 2 ** m)
            for a in range(dim):
                want = decasteljau([F(int(v)) for v in ctrl[c, :, a]], tf)
                assert got[c, j, a] == float(want), (d, c, k, a)


@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_oracle_equals_paper_seiler_forms(d):
    # Sec. 3.1 recursion with the closed-form difference terms, and the Sec. 4
    # texture layouts read at (t, st) / (t, st, st), reach the Bernstein value.
    rng = random.Random(7 + d)
    ctrl = _rand_int_ctrl(rng, 4, d, 2)
    ks = list(range(0, 65, 5)) + [64]
    t = np.array([k / 64 for k in ks])
    got = oracle.bezier(ctrl, t)
    for c in range(ctrl.shape[0]):
        for a in range(2):
            b = [F(int(v)) for v in ctrl[c, :, a]]
            tile = seiler_texture(b)
            for j, k in enumerate(ks):
                tf = F(k, 64)
                st = (1 - tf) * tf
                exact_value = bernstein_exact(b, tf)
                assert seiler_eval(b, tf) == exact_value
                if d <= 3:
                    tex = bilinear(tile[0], tf, st)
                else:
                    tex = trilinear(tile, tf, st, st)
                assert tex == exact_value
                assert float(exact_value) == got[c, j, a]


@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_peeled_seiler_terms_equal_paper_closed_forms(d):
    # The peeling reading used from degree 6 on reproduces the paper's closed
    # forms (Sec. 3.1) where those exist.
    from exact import seiler_terms_peel
    rng = random.Random(20 + d)
    for _ in range(5):
        b = [F(rng.randint(-8, 8)) for _ in range(d + 1)]
        paper = seiler_terms(b)
        peel = seiler_terms_peel(b)
        for k, v in paper.items():
            assert peel[k] == v, (d, k)


@pytest.mark.parametrize("d", [6, 7])
def test_degree_6_7_seiler_texture_equals_oracle(d):
    # 2x2x2 Seiler tile for degrees 6, 7 read at (t, 4 st, 16 st^2): exact
    # trilinear filtering reaches the Bernstein value (and the FP64 oracle),
    # and so does the Seiler recursion with the peeled terms.
    from exact import seiler_terms_peel, seiler_texture_quadratic_z
    rng = random.Random(30 + d)
    ctrl = _rand_int_ctrl(rng, 3, d, 2)
    ks = list(range(0, 65, 7)) + [64]
    got = oracle.bezier(ctrl, np.array([k / 64 for k in ks]))
    for c in range(ctrl.shape[0]):
        for a in range(2):
            b = [F(int(v)) for v in ctrl[c, :, a]]
            tile = seiler_texture_quadratic_z(b)
            terms = seiler_terms_peel(b)
            for j, k in enumerate(ks):
                tf = F(k, 64)
                st = (1 - tf) * tf
                exact_value = bernstein_exact(b, tf)
                assert seiler_eval(b, tf, terms) == exact_value
                assert trilinear(tile, tf, 4 * st, 16 * st * st) == exact_value
                assert float(exact_value) == got[c, j, a]


def test_paper_d2_formula_degenerates_at_cubic():
    # For d = 3 the Sec. 3.1 d_2 expression collapses to 0 for any control
    # points, so it must not be used there (the cubic uses d_{d-1} instead).
    from exact import seiler_d2
    rng = random.Random(3)
    for _ in range(20):
        b = [F(rng.randint(-9, 9)) for _ in range(4)]
        assert seiler_d2(b) == 0


def test_quartic_d2_formulas_agree():
    # At d = 4 both the d_2 and the d_{d-2} expressions name the same term.
    from exact import seiler_d2, seiler_dlast2
    rng = random.Random(4)
    for _ in range(20):
        b = [F(rng.randint(-9, 9)) for _ in range(5)]
        assert seiler_d2(b) == seiler_dlast2(b) == b[0] - 4 * b[1] + 6 * b[2] - 4 * b[3] + b[4]


def test_decasteljau_texture_cubic_equals_oracle():
    # Sec. 2: the 2x2x2 tile read at (t, t, t) gives the cubic point.
    rng = random.Random(11)
    ctrl = _rand_int_ctrl(rng, 5, 3, 3)
    ks = list(range(0, 33))
    got = oracle.bezier(ctrl, np.array([k / 32 for k in ks]))
    for c in range(5):
        for a in range(3):
            tile = decasteljau_texture([F(int(v)) for v in ctrl[c, :, a]])
            for j, k in enumerate(ks):
                tf = F(k, 32)
                assert float(trilinear(tile, tf, tf, tf)) == got[c, j, a]


def test_scipy_bpoly_agreement():
    from scipy.interpolate import BPoly
    rng = np.random.default_rng(5)
    for d in range(1, 9):
        ctrl = rng.uniform(-1, 1, size=(3, d + 1, 3))
        t = rng.uniform(0, 1, size=50)
        got = oracle.bezier(ctrl, t)
        for c in range(3):
            bp = BPoly(ctrl[c][:, None, :], [0.0, 1.0])
            np.testing.assert_allclose(got[c], bp(t), rtol=0, atol=1e-13)


def test_endpoints_partition_clamp_and_nan():
    rng = np.random.default_rng(6)
    for d in range(1, 9):
        ctrl = rng.uniform(-1, 1, size=(4, d + 1, 3)).astype(np.float32)
        got = oracle.bezier(ctrl, np.array([0.0, 1.0, -0.5, 1.5, np.nan]))
        np.testing.assert_array_equal(got[:, 0], ctrl[:, 0])
        np.testing.assert_array_equal(got[:, 1], ctrl[:, d])
        np.testing.assert_array_equal(got[:, 2], got[:, 0])  # clamped below
        np.testing.assert_array_equal(got[:, 3], got[:, 1])  # clamped above
        assert np.isnan(got[:, 4]).all()
        const = np.repeat(ctrl[:, :1], d + 1, axis=1)
        v = oracle.bezier(const, rng.uniform(0, 1, 40))
        np.testing.assert_allclose(v, np.repeat(ctrl[:, :1], 40, axis=1), rtol=0, atol=4e-16)


def test_degree_elevation_invariance():
    rng = np.random.default_rng(8)
    for d in range(1, 8):
        b = rng.uniform(-1, 1, size=(5, d + 1, 3))
        e = np.empty((5, d + 2, 3))
        e[:, 0] = b[:, 0]
        e[:, d + 1] = b[:, d]
        for i in range(1, d + 1):
            a = i / (d + 1)
            e[:, i] = a * b[:, i - 1] + (1 - a) * b[:, i]
        t = rng.uniform(0, 1, 64)
        np.testing.assert_allclose(oracle.bezier(b, t), oracle.bezier(e, t), rtol=0, atol=1e-14)


def test_grid_values_are_fp32_quotients():
    g = oracle.grid(256)
    want = (np.arange(256, dtype=np.float32) / np.float32(255)).astype(np.float64)
    np.testing.assert_array_equal(g, want)
    ctrl = np.random.default_rng(9).uniform(-1, 1, (3, 4, 3))
    np.testing.assert_array_equal(oracle.bezier_grid(ctrl, 256), oracle.bezier(ctrl, want))
    assert oracle.grid(1)[0] == 0.0


def test_rational_bezier_quarter_circle_golden():
    gold = json.load(open(os.path.join(GOLDEN, "quarter_circle_nurbs.json")))
    ctrl = np.array([gold["ctrl"]], np.float64)
    w = np.array([gold["weights"]])
    t = np.linspace(0, 1, 101)
    pts = oracle.bezier(ctrl, t, weights=w)
    np.testing.assert_allclose(np.linalg.norm(pts[0], axis=1), 1.0, rtol=0, atol=1e-15)
    pts3 = oracle.bezier(ctrl, np.array(gold["t"]), weights=w)
    np.testing.assert_allclose(pts3[0], np.array(gold["points"]), rtol=0, atol=1e-15)
    # scaling every weight by a constant leaves the curve unchanged
    np.testing.assert_allclose(oracle.bezier(ctrl, t, weights=3.5 * w), pts, rtol=0, atol=1e-15)
    # unit weights reduce to the integral curve
    np.testing.assert_allclose(oracle.bezier(ctrl, t, weights=np.ones_like(w)), oracle.bezier(ctrl, t),
                               rtol=0, atol=1e-15)


# ------------------------------------------------------------------ chains

def test_zigzag_golden_sizes():
    gold = json.load(open(os.path.join(GOLDEN, "zigzag_three_quadratics.json")))
    N = gold["n_segments"]
    P = [F(i * i - 3) for i in range(2 * N + 1)]
    T = zigzag_texture(P)
    assert len(T) == gold["texture_rows"] and len(T[0]) == gold["texture_columns"]
    assert 2 * N == gold["naive_columns"]
    assert len(T[0]) == gold["free_texels"] and N == gold["constraints"]


@pytest.mark.parametrize("free", [None, F(0), F(17, 3)])
def test_oracle_chain_equals_zigzag_texture(free):
    # Eq. 1-2: any choice of the free texel gives the same chain, and the
    # zig-zag texture read along its path equals the oracle's segment sum.
    rng = random.Random(12)
    N, dim = 5, 2
    P = [[F(rng.randint(-8, 8)) for _ in range(dim)] for _ in range(2 * N + 1)]
    ctrl = np.array([[[float(v) for v in p] for p in P]])
    ts = [F(k, 16) for k in range(0, 16 * N + 1)]
    got = oracle.chain(ctrl, N, 2, np.array([float(x) for x in ts]))
    for a in range(dim):
        T = zigzag_texture([p[a] for p in P], t0=free)
        for j, tf in enumerate(ts):
            assert float(zigzag_sample(T, tf)) == got[0, j, a]


@pytest.mark.parametrize("free", [(None, None, None), (F(3), F(-7, 2), None), (F(0), F(0), "random")])
def test_oracle_cubic_chain_equals_zigzag3_texture(free):
    # Sec. 2.1, last paragraph (cubic C0 chains from quadratic chains placed
    # front to back in a 3D texture): the (N+1) x 2 x 2 texture of
    # zigzag3_texture, read trilinearly along its zig-zag path, equals the
    # oracle's cubic chain for any choice of the free texels
    rng = random.Random(31)
    N, dim = 5, 2
    P = [[F(rng.randint(-8, 8)) for _ in range(dim)] for _ in range(3 * N + 1)]
    ctrl = np.array([[[float(v) for v in p] for p in P]])
    ts = [F(k, 16) for k in range(0, 16 * N + 1)]
    got = oracle.chain(ctrl, N, 3, np.array([float(x) for x in ts]))
    s0, d0, split = free
    for a in range(dim):
        sp = [F(rng.randint(-5, 5), 3) for _ in range(N + 1)] if split == "random" else None
        T = zigzag3_texture([p[a] for p in P], s0=s0, d0=d0, split=sp)
        for j, tf in enumerate(ts):
            assert float(zigzag3_sample(T, tf)) == got[0, j, a]


def test_zigzag3_slices_are_quadratic_zigzag_chains():
    # each z slice of the cubic texture, read bilinearly along the 2D
    # zig-zag path, is a C0 chain of quadratics (the "two quadratic chains
    # front to back"), and lerping the slice read that starts at a segment's
    # corner with the other one gives the cubic
    rng = random.Random(32)
    N = 6
    P = [F(rng.randint(-8, 8)) for _ in range(3 * N + 1)]
    T = zigzag3_texture(P, s0=F(1), d0=F(-2))
    ts = [F(k, 8) for k in range(0, 8 * N + 1)]
    for zs in range(2):
        sl = T[zs]
        vals = {}
        for tf in ts:
            k = min(int(tf), N - 1)
            tau = tf - k
            y = tau if k % 2 == 0 else 1 - tau
            tile = [[sl[0][k], sl[0][k + 1]], [sl[1][k], sl[1][k + 1]]]
            vals.setdefault(tf, []).append(bilinear(tile, tau, y))
        # continuity at the joints: segment k at tau = 1 meets segment k+1 at tau = 0
        for k in range(1, N):
            left = bilinear([[sl[0][k - 1], sl[0][k]], [sl[1][k - 1], sl[1][k]]], F(1), F(1) if (k - 1) % 2 == 0 else F(0))
            right = bilinear([[sl[0][k], sl[0][k + 1]], [sl[1][k], sl[1][k + 1]]], F(0), F(0) if k % 2 == 0 else F(1))
            assert left == right
    for tf in ts:
        k = min(int(tf), N - 1)
        tau = tf - k
        y = tau if k % 2 == 0 else 1 - tau
        front, back = (T[0], T[1]) if k % 2 == 0 else (T[1], T[0])
        qf = bilinear([[front[0][k], front[0][k + 1]], [front[1][k], front[1][k + 1]]], tau, y)
        qb = bilinear([[back[0][k], back[0][k + 1]], [back[1][k], back[1][k + 1]]], tau, y)
        assert lerp(qf, qb, tau) == bernstein_exact(P[3 * k:3 * k + 4], tau)


def test_segment_quadratics_front_to_back_are_not_a_c0_chain():
    # the literal reading -- the front slice holding each segment's own
    # quadratic (P_3k, P_3k+1, P_3k+2) and the back slice (P_3k+1, P_3k+2,
    # P_3k+3), as in the single-cubic tile of Sec. 2 -- needs consecutive
    # front quadratics to meet (P_3k+2 == P_3k+3), which a general cubic chain
    # violates, so those quadratics cannot share zig-zag columns; the
    # construction above stores other quadratics whose z-lerp is the cubic
    P = [F(v) for v in (0, 3, -2, 5, 1, 4, -1)]           # two cubic segments
    front_end_0, front_start_1 = P[2], P[3]
    back_end_0, back_start_1 = P[3], P[4]
    assert front_end_0 != front_start_1 and back_end_0 != back_start_1


def test_chain_continuity_and_segments():
    rng = np.random.default_rng(13)
    N, p = 7, 3
    ctrl = rng.uniform(-1, 1, size=(2, N * p + 1, 3))
    t = np.arange(N + 1, dtype=np.float64)
    got = oracle.chain(ctrl, N, p, t)
    np.testing.assert_array_equal(got[:, :, :], ctrl[:, ::p, :])
    tt = np.array([2.25, 6.75])
    got2 = oracle.chain(ctrl, N, p, tt)
    seg2 = oracle.bezier(ctrl[:, 6:10], np.array([0.25]))
    seg6 = oracle.bezier(ctrl[:, 18:22], np.array([0.75]))
    np.testing.assert_allclose(got2[:, 0], seg2[:, 0], atol=1e-15)
    np.testing.assert_allclose(got2[:, 1], seg6[:, 0], atol=1e-15)


# ------------------------------------------------------------------ polyline

def test_polyline_length_line_and_bound():
    rng = np.random.default_rng(14)
    b = rng.uniform(-1, 1, size=(4, 2, 3))
    t = np.sort(np.concatenate([[0.0, 1.0], rng.uniform(0, 1, 30)]))
    L = oracle.polyline_length(oracle.bezier(b, t))
    np.testing.assert_allclose(L, np.linalg.norm(b[:, 1] - b[:, 0], axis=1), rtol=1e-14)
    # a polyline inscribed in a curve is never longer than the curve and
    # converges to its arc length (quadrature of |C'| from SciPy's BPoly)
    from scipy.integrate import quad
    from scipy.interpolate import BPoly
    c = rng.uniform(-1, 1, size=(1, 4, 3))
    bp = BPoly(c[0][:, None, :], [0.0, 1.0]).derivative()
    arc = quad(lambda s: np.linalg.norm(bp(s)), 0, 1, epsabs=1e-13, limit=200)[0]
    prev = 0.0
    for n in (8, 64, 512, 4096):
        Ln = oracle.polyline_length(oracle.bezier(c, np.linspace(0, 1, n)))[0]
        assert prev <= Ln <= arc + 1e-12
        prev = Ln
    assert arc - prev < 1e-5


def test_hash_parameters_uniform_and_fp32_exact():
    t = oracle.hash_t(20260316, 1, 0, 64, 1024)
    assert t.min() >= 0.0 and t.max() < 1.0
    np.testing.assert_array_equal(t, t.astype(np.float32).astype(np.float64))
    assert abs(t.mean() - 0.5) < 0.005
    # Kolmogorov-Smirnov against U[0,1)
    from scipy.stats import kstest
    assert kstest(t.ravel(), "uniform").pvalue > 1e-4
    # chunked generation (curve offset) equals one-shot generation
    np.testing.assert_array_equal(oracle.hash_t(20260316, 1, 10, 5, 1024), t[10:15])
    # lowbias32 is a bijection on 32-bit words: invert it by undoing each step
    M = 2 ** 32
    inv1, inv2 = pow(0x7FEB352D, -1, M), pow(0x846CA68B, -1, M)

    def unxorshift(y, s):
        x = y
        for _ in range(32 // s + 1):
            x = y ^ (x >> s)
        return x

    for x in [0, 1, 2, 12345, 0xDEADBEEF, 0xFFFFFFFF]:
        y = oracle.lowbias32(x)
        y = unxorshift(y, 16)
        y = (y * inv2) % M
        y = unxorshift(y, 15)
        y = (y * inv1) % M
        y = unxorshift(y, 16)
        assert y == x


def test_hash_avalanche():
    # a property of the mixer rather than its formula: flipping any one input
    # bit flips every output bit with probability close to 1/2 (a weak or
    # mistyped multiplier leaves some bit pairs far from it); 4096 random
    # inputs, so the sampling error of each probability is about 0.008
    rng = np.random.default_rng(15)
    xs = [int(v) for v in rng.integers(0, 2 ** 32, 4096, dtype=np.uint64)]
    base = np.array([oracle.lowbias32(x) for x in xs], np.uint64)
    p = np.zeros((32, 32))
    for i in range(32):
        flipped = np.array([oracle.lowbias32(x ^ (1 << i)) for x in xs], np.uint64)
        diff = base ^ flipped
        p[i] = [(((diff >> np.uint64(j)) & np.uint64(1)).astype(np.float64)).mean() for j in range(32)]
    assert np.abs(p - 0.5).max() < 0.05, np.abs(p - 0.5).max()
