"""Exact rational constructions used to pin the FP64 oracle.

Each routine here reaches a curve value by a route *different* from the
oracle's Bernstein sum / Cox-de Boor recursion, in ``fractions.Fraction``
arithmetic so that no rounding is involved:

* ``decasteljau`` -- recursive linear interpolation (paper Sec. 2).
* ``seiler_*`` -- the paper's Seiler recursion and difference terms (Sec. 3.1)
  and its pure-lerp / texture forms (Sec. 4, Eq. 3-6 and the layout table).
* ``bilinear`` / ``trilinear`` -- exact linear texture filtering of a 2x2 or
  2x2x2 tile at fractional position (the arithmetic the texture unit is meant
  to perform, without weight quantisation).
* ``zigzag_*`` -- the C0 chain texture of Sec. 2.1 (Eq. 1-2, Fig. 2).
* ``boehm_*`` -- Boehm knot insertion, turning a B-spline into Bezier spans
  (Sec. 2.2 names it as the route from B-splines to Bezier curves).
"""
from fractions import Fraction as F
from math import comb


def lerp(a, b, t):
    return a + (b - a) * t


def decasteljau(b, t):
    """Point of the Bezier curve with control values b (scalars) at t."""
    pts = list(b)
    while len(pts) > 1:
        pts = [lerp(pts[i], pts[i + 1], t) for i in range(len(pts) - 1)]
    return pts[0]


def bernstein_exact(b, t):
    d = len(b) - 1
    return sum(comb(d, i) * (1 - t) ** (d - i) * t ** i * b[i] for i in range(d + 1))


# ------------------------------------------------------------- Seiler (Sec. 3)

def seiler_d1(b):
    d = len(b) - 1
    return d * (b[1] - b[0]) - (b[d] - b[0])


def seiler_dlast(b):
    d = len(b) - 1
    return d * (b[d - 1] - b[d]) - (b[0] - b[d])


def seiler_d2(b):
    """The paper's d_2 for degrees up to 5 (Sec. 3.1)."""
    d = len(b) - 1
    return (comb(d, 2) * (b[2] - b[1]) - comb(d - 2, 2) * (b[1] - b[0])
            - (d - 3) * (b[d - 1] - b[d]) - 3 * (b[d - 1] - b[1]))


def seiler_dlast2(b):
    """The paper's d_{d-2} for degrees up to 5 (Sec. 3.1)."""
    d = len(b) - 1
    return (comb(d, 2) * (b[d - 2] - b[d - 1]) - comb(d - 2, 2) * (b[d - 1] - b[d])
            - (d - 3) * (b[1] - b[0]) - 3 * (b[1] - b[d - 1]))


def seiler_terms(b):
    """Difference terms {i: d_i} from the paper's closed forms, degree 1..5."""
    d = len(b) - 1
    terms = {}
    if d >= 2:
        terms[1] = seiler_d1(b)
        terms[d - 1] = seiler_dlast(b)
    if d in (4, 5):
        terms[2] = seiler_d2(b)
        terms[d - 2] = seiler_dlast2(b)
    return terms


def seiler_eval(b, t, terms=None):
    """C(t) = L(b0, bd, t) + (1-t) t D_1(t), D_i by the paper's three cases."""
    d = len(b) - 1
    dd = seiler_terms(b) if terms is None else terms
    st = (1 - t) * t

    def D(i):
        if 2 * i == d + 1:
            return 0
        if 2 * i == d:
            return dd[i]
        return lerp(dd[i], dd[d - i], t) + st * D(i + 1)

    if d == 1:
        return lerp(b[0], b[1], t)
    return lerp(b[0], b[d], t) + st * D(1)


def seiler_terms_peel(b):
    """Difference terms {k: d_k} of the Seiler form for any degree, by exact
    polynomial division (sympy): P_0 = C; d_k = P_k(0), d_(d-k) = P_k(1) and
    P_(k+1) = (P_k - L(P_k(0), P_k(1), t)) / (t (1 - t)), which is exact since
    the numerator vanishes at t = 0 and t = 1.  For degrees <= 5 the result
    equals the paper's closed forms (pinned by a test)."""
    import sympy
    t = sympy.symbols("t")
    d = len(b) - 1
    P = sum(sympy.Rational(comb(d, i)) * (1 - t) ** (d - i) * t ** i * sympy.Rational(b[i].numerator, b[i].denominator)
            for i in range(d + 1))
    P = sympy.expand(P)
    terms = {}
    k = 0
    m = d
    while m >= 0:
        lo, hi = P.subs(t, 0), P.subs(t, 1)
        terms[k] = F(int(lo.p), int(lo.q))
        terms[d - k] = F(int(hi.p), int(hi.q))
        if m < 2:
            break
        q, r = sympy.div(sympy.expand(P - (lo + (hi - lo) * t)), sympy.expand(t * (1 - t)), t)
        assert r == 0
        P = sympy.expand(q)
        k += 1
        m -= 2
    return terms


def seiler_texture_quadratic_z(b):
    """2x2x2 tile for degrees 6, 7 read at (t, 4 st, 16 st^2) (a derivation
    beyond the paper's layout table): trilinear filtering of tile[z][y][x] at
    (x, y, z) is L0(x) + y (L1 - L0) + z (L2 - L0) + yz (...), so with
    L_k(t) = L(d_k, d_(d-k), t) and texels
      z=0: [[d0, dd], [d0 + d1/4, dd + d_(d-1)/4]]
      z=1: [[d0 + d2/16, dd + d_(d-2)/16],
            [d0 + d1/4 + d2/16 + d3/64, dd + d_(d-1)/4 + d_(d-2)/16 + d_(d-3)/64]]
    the read gives L0 + st L1 + st^2 L2 + st^3 L3, the Seiler form of degree
    <= 7 (d_0 = b_0, d_d = b_d)."""
    d = len(b) - 1
    assert d in (6, 7)
    dd = seiler_terms_peel(b)
    lo = [dd[k] for k in range(4)]
    hi = [dd[d - k] for k in range(4)]
    z0 = [[lo[0], hi[0]], [lo[0] + lo[1] / 4, hi[0] + hi[1] / 4]]
    z1 = [[lo[0] + lo[2] / 16, hi[0] + hi[2] / 16],
          [lo[0] + lo[1] / 4 + lo[2] / 16 + lo[3] / 64, hi[0] + hi[1] / 4 + hi[2] / 16 + hi[3] / 64]]
    return [z0, z1]


def bilinear(tile, x, y):
    """tile[y][x] (2x2), fractional weights x, y in [0,1]."""
    return lerp(lerp(tile[0][0], tile[0][1], x), lerp(tile[1][0], tile[1][1], x), y)


def trilinear(tile, x, y, z):
    """tile[z][y][x] (2x2x2)."""
    return lerp(bilinear(tile[0], x, y), bilinear(tile[1], x, y), z)


def seiler_texture(b):
    """Texel contents of the paper's Seiler layout table (degrees 2..5):
    tile[z][y][x]; one z slice for degrees 2, 3 (read at (t, st)), two for
    degrees 4, 5 (read at (t, st, st))."""
    d = len(b) - 1
    dd = seiler_terms(b)
    if d == 2:
        return [[[b[0], b[2]], [b[0] + dd[1], b[2] + dd[1]]]]
    if d == 3:
        return [[[b[0], b[3]], [b[0] + dd[1], b[3] + dd[2]]]]
    if d in (4, 5):
        z0 = [[b[0], b[d]], [b[0], b[d]]]
        z1 = [[b[0] + dd[1], b[d] + dd[d - 1]],
              [b[0] + dd[1] + dd[2], b[d] + dd[d - 1] + dd[d - 2]]]
        return [z0, z1]
    raise ValueError("layout defined for degrees 2..5")


def decasteljau_texture(b):
    """2x2x2 tile for a cubic: z=0 holds the quadratic (b0,b1,b2) as
    [[b0,b1],[b1,b2]], z=1 the quadratic (b1,b2,b3) (Sec. 2)."""
    assert len(b) == 4
    return [[[b[0], b[1]], [b[1], b[2]]], [[b[1], b[2]], [b[2], b[3]]]]


# ------------------------------------------------------------- zig-zag (Sec. 2.1)

def zigzag_texture(P, t0=None):
    """Two-row texture T[row][col], (N+1) columns, for a C0 chain of N
    quadratics with logical control points P[0..2N].

    Segment k is read between texel (k, r_k) and (k+1, 1-r_k), r_k = k mod 2,
    which hold the segment end points; the two other texels of the 2x2 window
    must average to the middle control point P[2k+1] (Eq. 1-2).  Those free
    texels form a sequence F_0..F_N with F_k + F_{k+1} = 2 P[2k+1]: N
    constraints, N+1 unknowns, so F_0 (= t0, default P[1]) is free."""
    N = (len(P) - 1) // 2
    T = [[None] * (N + 1), [None] * (N + 1)]
    Fk = P[1] if t0 is None else t0
    for k in range(N + 1):
        T[k % 2][k] = P[2 * k]            # end point of segment k-1 / start of k
        T[1 - k % 2][k] = Fk              # free texel in column k
        if k < N:
            Fk = 2 * P[2 * k + 1] - Fk
    return T


def zigzag_sample(T, t):
    """Sample the chain texture at global t in [0, N] along the zig-zag path:
    segment k, local tau; x weight tau between columns k, k+1; y weight
    tau for even k (row 0 -> row 1) and 1 - tau for odd k."""
    N = len(T[0]) - 1
    k = min(int(t), N - 1)
    tau = t - k
    y = tau if k % 2 == 0 else 1 - tau
    tile = [[T[0][k], T[0][k + 1]], [T[1][k], T[1][k + 1]]]
    return bilinear(tile, tau, y)


# ------------------------------------------------------------- cubic zig-zag (Sec. 2.1, last paragraph)

def zigzag3_texture(P, s0=None, d0=None, split=None):
    """Texture T[z][y][col], 2 x 2 x (N+1), for a C0 chain of N cubics with
    logical control points P[0..3N], read trilinearly along a 3D zig-zag.

    Column k has the corner c_k = (y, z) = (k mod 2, k mod 2), which holds
    P[3k]; the texel with y flipped (a_k), with z flipped (b_k) and with
    both flipped (d_k) are free.  Trilinear filtering of the window of
    columns k, k+1 read from corner c_k at (tau, tau, tau) weighs a texel by
    tau^m (1 - tau)^(3-m), m its number of flips away from the corner, so
    the window evaluates the cubic whose control points are the class means:
    P[3k] (m = 0), (a_k + b_k + d_(k+1)) / 3 (m = 1), (d_k + a_(k+1) +
    b_(k+1)) / 3 (m = 2), P[3k+3] (m = 3) -- the three-texel analogue of
    E = (B + C) / 2 (Eq. 1-2).  With s_k = a_k + b_k the 2N constraints are
    d_(k+1) = 3 P[3k+1] - s_k and s_(k+1) = 3 P[3k+2] - d_k on 2 (N+1)
    unknowns: s_0, d_0 are free, and so is how each s_k splits into a_k,
    b_k (split[k] = a_k - s_k / 2, default 0)."""
    N = (len(P) - 1) // 3
    s = [None] * (N + 1)
    d = [None] * (N + 1)
    s[0] = 2 * P[1] if s0 is None else s0
    d[0] = P[2] if d0 is None else d0
    for k in range(N):
        d[k + 1] = 3 * P[3 * k + 1] - s[k]
        s[k + 1] = 3 * P[3 * k + 2] - d[k]
    T = [[[None] * (N + 1) for _ in range(2)] for _ in range(2)]
    for k in range(N + 1):
        c = k % 2
        e = 0 if split is None else split[k]
        a = s[k] / 2 + e
        b = s[k] - a
        T[c][c][k] = P[3 * k]
        T[c][1 - c][k] = a            # y flipped
        T[1 - c][c][k] = b            # z flipped
        T[1 - c][1 - c][k] = d[k]     # both flipped
    return T


def zigzag3_sample(T, t):
    """Trilinear read of the cubic zig-zag texture at global t in [0, N]:
    segment k, local tau; x weight tau between columns k, k+1; y and z
    weights tau on even segments (from row / slice 0) and 1 - tau on odd."""
    N = len(T[0][0]) - 1
    k = min(int(t), N - 1)
    tau = t - k
    w = tau if k % 2 == 0 else 1 - tau
    tile = [[[T[z][y][k], T[z][y][k + 1]] for y in range(2)] for z in range(2)]
    return trilinear(tile, tau, w, w)


# ------------------------------------------------------------- Boehm (Sec. 2.2)

def boehm_insert(U, P, p, u):
    """Insert knot u once (Boehm's algorithm).  U list of knots, P list of
    control values.  Returns (U', P')."""
    n = len(P)
    k = max(i for i in range(p, n) if U[i] <= u < U[i + 1]) if u < U[n] else n - 1
    Q = []
    for i in range(n + 1):
        if i <= k - p:
            Q.append(P[i])
        elif i > k:
            Q.append(P[i - 1])
        else:
            a = (u - U[i]) / (U[i + p] - U[i])
            Q.append((1 - a) * P[i - 1] + a * P[i])
    return U[: k + 1] + [u] + U[k + 1:], Q


def boehm_to_bezier(U, P, p):
    """Insert every interior knot up to multiplicity p, giving Bezier spans.
    Returns a list of (u_start, u_end, [p+1 control values])."""
    U = list(U)
    P = list(P)
    interior = sorted(set(U[p + 1: len(P)]))
    for u in interior:
        while U.count(u) < p:
            U, P = boehm_insert(U, P, p, u)
    breaks = sorted(set(U))
    spans = []
    for s in range(len(breaks) - 1):
        spans.append((breaks[s], breaks[s + 1], P[s * p: s * p + p + 1]))
    return spans


def bspline_via_boehm(U, P, p, u):
    """B-spline value at u via Boehm extraction + de Casteljau on the span."""
    spans = boehm_to_bezier(U, P, p)
    for a, b_, Q in spans:
        if a <= u < b_ or (u == b_ and b_ == spans[-1][1]):
            return decasteljau(Q, (u - a) / (b_ - a))
    raise ValueError("u outside the domain")


def clamped_uniform_knots_exact(n, p):
    return [F(0)] * (p + 1) + [F(i, n - p) for i in range(1, n - p)] + [F(1)] * (p + 1)
