// curve_eval.cuh -- register evaluators for Bezier curves and the kernels that
// drive them: one curve per warp (every variant), and for the fused
// evaluate-and-measure form of centred Horner on 3D curves of degree <= 4 two
// curves per warp (k_curve_pair) or 8 / 4 lanes per curve (k_curve_group).
//
// Each evaluator is a struct with setup(b) (per curve, once) and eval(t, P)
// (per parameter).  D is the degree when known at compile time, or 0 for the
// runtime-degree fallback (degree <= kMaxDegree).  DIM is the point dimension.
//
//   Horner          power basis about t = 0 (paper Sec. 2.2: power basis <->
//                   Bernstein); coefficients a_k = binom(d,k) Delta^k b_0.
//   HornerCentred   power basis about t = 1/2; c_k = binom(d,k) times the
//                   Bernstein value at 1/2 of the k-th forward differences.
//   Bernstein       sum_i binom(d,i) (1-t)^(d-i) t^i b_i ("Polynomial" of Sec. 5).
//   DeCasteljau     d(d+1)/2 lerps at the same t (Sec. 2).
//   Seiler          C = L(b0, bd, t) + st D_1, D_i = L(d_i, d_(d-i), t) + st D_(i+1)
//                   (Sec. 3.1); d_i from the closed forms for degree <= 5 and
//                   by exact peeling of the s-power form above that.
//
// Setup runs in FP32 up to degree 7 and in FP64 from degree 8 on, except the
// centred power basis, whose FP32 conversion alone costs more than 1e-6 of
// the curve diagonal at degree 7 (1.4e-6 measured); it switches to FP64 at
// degree 5.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace bez {

constexpr int kFp64Setup = 8;         // power basis about 0, Seiler peeling
constexpr int kFp64SetupCentred = 5;  // power basis about 1/2

template <int D>
struct Deg {
    __device__ __forceinline__ static int get(int) { return D; }
    static constexpr int N = D + 1;  // array extent
};
template <>
struct Deg<0> {
    __device__ __forceinline__ static int get(int d) { return d; }
    static constexpr int N = kMaxDegree + 1;
};

// ---------------------------------------------------------------- setup helpers

// Forward differences of b (degree d) in place: after the call
// w[k] = Delta^k b_0 for k = 0..d.  Templated on the arithmetic type S.
template <typename S, int N>
__device__ __forceinline__ void forward_differences_at0(S (&w)[N], int d)
{
#pragma unroll
    for (int k = 1; k < N; ++k) {
        if (k > d) break;
#pragma unroll
        for (int i = N - 1; i >= 1; --i)
            if (i >= k && i <= d) w[i] = w[i] - w[i - 1];
    }
}

// ---------------------------------------------------------------- centred basis matrix

// T_d[m][i]: coefficient of b_i in the power coefficient about t = 1/2,
// c_m = sum_i T_d[m][i] b_i = binom(d, m) * (Bernstein value at 1/2 of the
// m-th forward differences) -- the conversion applied to unit vectors.  The
// entries are small integers over powers of two (exact in FP32 and FP64).
struct CentredTables {
    double t[8][8][8];  // [d][m][i], d = 1..7
};
constexpr CentredTables make_centred_tables()
{
    CentredTables r{};
    for (int d = 1; d <= 7; ++d)
        for (int i = 0; i <= d; ++i) {
            double w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            w[i] = 1.0;
            double bin = 1.0;
            for (int m = 0; m <= d; ++m) {
                double h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                for (int k = 0; k <= d - m; ++k) h[k] = w[k];
                for (int q = 1; q <= d - m; ++q)
                    for (int k = 0; k <= d - m - q; ++k) h[k] = 0.5 * (h[k] + h[k + 1]);
                r.t[d][m][i] = bin * h[0];
                bin = bin * (double)(d - m) / (double)(m + 1);
                for (int k = 0; k < d - m; ++k) w[k] = w[k + 1] - w[k];
            }
        }
    return r;
}
static __constant__ CentredTables kCentredT = make_centred_tables();

// ---------------------------------------------------------------- evaluators

template <int VAR, int D, int DIM>
struct Eval;

template <int D, int DIM>
struct Eval<VAR_HORNER, D, DIM> {
    static constexpr int N = Deg<D>::N;
    float a[N][DIM];
    int d;
    template <typename S>
    __device__ __forceinline__ void setup_t(const float (&b)[N][DIM])
    {
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            S w[N];
#pragma unroll
            for (int i = 0; i < N; ++i) w[i] = (i <= d) ? (S)b[i][k] : (S)0;
            forward_differences_at0<S, N>(w, d);
            S bin = 1;  // binom(d, i) built incrementally
#pragma unroll
            for (int i = 0; i < N; ++i) {
                if (i <= d) a[i][k] = (float)(bin * w[i]);
                bin = bin * (S)(d - i) / (S)(i + 1);
            }
        }
    }
    __device__ __forceinline__ void setup(const float (&b)[N][DIM], int deg)
    {
        d = Deg<D>::get(deg);
        if (d >= kFp64Setup) setup_t<double>(b);
        else setup_t<float>(b);
    }
    __device__ __forceinline__ void eval(float t, float (&P)[DIM]) const
    {
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            float acc = a[N - 1][k];
            if (D == 0) acc = a[d][k];
#pragma unroll
            for (int i = N - 2; i >= 0; --i)
                if (i < d) acc = fmaf(acc, t, a[i][k]);
            P[k] = acc;
        }
    }
};

template <int D, int DIM>
struct Eval<VAR_HORNER_CENTRED, D, DIM> {
    static constexpr int N = Deg<D>::N;
    float a[N][DIM];
    int d;
    template <typename S>
    __device__ __forceinline__ void setup_t(const float (&b)[N][DIM])
    {
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            S w[N];
#pragma unroll
            for (int i = 0; i < N; ++i) w[i] = (i <= d) ? (S)b[i][k] : (S)0;
            S bin = 1;
#pragma unroll
            for (int m = 0; m < N; ++m) {
                if (m > d) break;
                // w[0..d-m] holds Delta^m b; its Bernstein value at 1/2 by halving
                S h[N];
#pragma unroll
                for (int i = 0; i < N; ++i) h[i] = w[i];
#pragma unroll
                for (int r = 1; r < N; ++r)
#pragma unroll
                    for (int i = 0; i < N - 1; ++i)
                        if (r <= d - m && i <= d - m - r) h[i] = (S)0.5 * (h[i] + h[i + 1]);
                a[m][k] = (float)(bin * h[0]);
                bin = bin * (S)(d - m) / (S)(m + 1);
#pragma unroll
                for (int i = 0; i < N - 1; ++i)
                    if (i < d - m) w[i] = w[i + 1] - w[i];
            }
        }
    }
    __device__ __forceinline__ void setup(const float (&b)[N][DIM], int deg)
    {
        d = Deg<D>::get(deg);
        if (d >= kFp64SetupCentred) setup_t<double>(b);
        else setup_t<float>(b);
    }
    // Warp-cooperative setup for 3D curves of fixed degree: the curve's
    // control points are spread one element per lane (lane 3i + k holds
    // b_i[k], in v); lane 3m + k forms a[m][k] = sum_i T_d[m][i] b_i[k] (FP64
    // from degree 5, like setup) and the warp broadcasts the coefficients.
    // One dot product per lane instead of the whole conversion per lane.
    // base: first lane of the group holding the curve (0 for a whole warp;
    // 0 or 16 when two curves share a warp)
    __device__ __forceinline__ void setup_warp(float v, int lane, int base = 0)
    {
        static_assert(D > 0 && DIM == 3 && 3 * (D + 1) <= 32, "fixed-degree 3D curves only");
        d = D;
        using S = typename std::conditional<(D >= kFp64SetupCentred), double, float>::type;
        const int li = lane - base;
        const int m = li < 3 * (D + 1) ? li / 3 : 0;
        const int k = li < 3 * (D + 1) ? li - 3 * m : 0;
        S acc = (S)0;
#pragma unroll
        for (int i = 0; i <= D; ++i) {
            const float bik = __shfl_sync(kFull, v, base + 3 * i + k);
            acc = fma((S)kCentredT.t[D][m][i], (S)bik, acc);
        }
        const float cm = (float)acc;
#pragma unroll
        for (int mm = 0; mm <= D; ++mm)
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) a[mm][kk] = __shfl_sync(kFull, cm, base + 3 * mm + kk);
    }
    // Setup for 3D curves of fixed degree held by a group of G lanes (lane
    // base + r, slot s of v holds element G s + r of the curve, b_i[k] being
    // element 3 i + k): every lane gathers the 3 (D + 1) elements and forms
    // all coefficients itself.  The operator entries are then the same for
    // every lane (uniform constant reads), and the sums run in setup_warp's
    // order, so the coefficients are the same as setup_warp's.
    template <int G, int NL>
    __device__ __forceinline__ void setup_group(const float (&v)[NL], int base)
    {
        static_assert(D > 0 && DIM == 3 && 3 * (D + 1) <= G * NL, "fixed-degree 3D curves only");
        d = D;
        using S = typename std::conditional<(D >= kFp64SetupCentred), double, float>::type;
        float b[D + 1][3];
#pragma unroll
        for (int i = 0; i <= D; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int e = 3 * i + k;
                b[i][k] = __shfl_sync(kFull, v[e / G], base + e % G);
            }
#pragma unroll
        for (int m = 0; m <= D; ++m)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                S acc = (S)0;
#pragma unroll
                for (int i = 0; i <= D; ++i) acc = fma((S)kCentredT.t[D][m][i], (S)b[i][k], acc);
                a[m][k] = (float)acc;
            }
    }
    __device__ __forceinline__ void eval(float t, float (&P)[DIM]) const { eval_u(t - 0.5f, P); }
    // evaluate at u = t - 1/2
    __device__ __forceinline__ void eval_u(float u, float (&P)[DIM]) const
    {
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            float acc = a[N - 1][k];
            if (D == 0) acc = a[d][k];
#pragma unroll
            for (int i = N - 2; i >= 0; --i)
                if (i < d) acc = fmaf(acc, u, a[i][k]);
            P[k] = acc;
        }
    }
};

template <int D, int DIM>
struct Eval<VAR_BERNSTEIN, D, DIM> {
    static constexpr int N = Deg<D>::N;
    float p[N][DIM];  // binom(d,i) b_i
    int d;
    __device__ __forceinline__ void setup(const float (&b)[N][DIM], int deg)
    {
        d = Deg<D>::get(deg);
        float bin = 1.f;
#pragma unroll
        for (int i = 0; i < N; ++i) {
#pragma unroll
            for (int k = 0; k < DIM; ++k) p[i][k] = bin * b[i][k];
            bin = bin * (float)(d - i) / (float)(i + 1);
        }
    }
    __device__ __forceinline__ void eval(float t, float (&P)[DIM]) const
    {
        const float s = 1.0f - t;
        float tp[N], sp[N];
        tp[0] = 1.f;
        sp[0] = 1.f;
#pragma unroll
        for (int i = 1; i < N; ++i) {
            tp[i] = tp[i - 1] * t;
            sp[i] = sp[i - 1] * s;
        }
#pragma unroll
        for (int k = 0; k < DIM; ++k) P[k] = 0.f;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            if (i > d) break;
            const float B = (D == 0) ? tp[i] * sp[d - i] : tp[i] * sp[N - 1 - i];
#pragma unroll
            for (int k = 0; k < DIM; ++k) P[k] = fmaf(B, p[i][k], P[k]);
        }
    }
};

template <int D, int DIM>
struct Eval<VAR_DECASTELJAU, D, DIM> {
    static constexpr int N = Deg<D>::N;
    float b[N][DIM];
    int d;
    __device__ __forceinline__ void setup(const float (&bb)[N][DIM], int deg)
    {
        d = Deg<D>::get(deg);
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int k = 0; k < DIM; ++k) b[i][k] = bb[i][k];
    }
    __device__ __forceinline__ void eval(float t, float (&P)[DIM]) const
    {
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            float w[N];
#pragma unroll
            for (int i = 0; i < N; ++i) w[i] = b[i][k];
#pragma unroll
            for (int r = 1; r < N; ++r)
#pragma unroll
                for (int i = 0; i < N - 1; ++i)
                    if (r <= d && i <= d - r) w[i] = lerp(w[i], w[i + 1], t);
            P[k] = w[0];
        }
    }
};

// Seiler difference terms.  lo[k] = d_k, hi[k] = d_(d-k) for k = 0..floor(d/2)
// (lo[0] = b_0, hi[0] = b_d).
template <int D, int DIM>
struct Eval<VAR_SEILER, D, DIM> {
    static constexpr int N = Deg<D>::N;
    static constexpr int H = N / 2 + 1;
    float lo[H][DIM], hi[H][DIM];
    int d;

    // closed forms of Sec. 3.1 (valid for d <= 5)
    __device__ __forceinline__ void setup_closed(const float (&b)[N][DIM])
    {
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const float b0 = b[0][k], bd = b[d][k];
            lo[0][k] = b0;
            hi[0][k] = bd;
            if (d >= 2) {
                const float fd = (float)d;
                lo[1][k] = fd * (b[1][k] - b0) - (bd - b0);
                hi[1][k] = fd * (b[d - 1][k] - bd) - (b0 - bd);
            }
            if (H > 2 && d >= 4) {
                const float c2 = (float)(d * (d - 1) / 2), c2m = (float)((d - 2) * (d - 3) / 2);
                const float e = (float)(d - 3);
                lo[2][k] = c2 * (b[2][k] - b[1][k]) - c2m * (b[1][k] - b0) - e * (b[d - 1][k] - bd) -
                           3.f * (b[d - 1][k] - b[1][k]);
                hi[2][k] = c2 * (b[d - 2][k] - b[d - 1][k]) - c2m * (b[d - 1][k] - bd) - e * (b[1][k] - b0) -
                           3.f * (b[1][k] - b[d - 1][k]);
            }
        }
    }

    // Any degree: peel P = L(P(0), P(1), t) + t(1-t) Q repeatedly in the
    // Bernstein basis; Q has coefficients q_(j+1) m(m-1)/((j+1)(m-1-j)) where
    // q_i = c_i - ((1 - i/m) c_0 + (i/m) c_m).
    template <typename S>
    __device__ __forceinline__ void setup_peel(const float (&b)[N][DIM])
    {
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            S c[N];
#pragma unroll
            for (int i = 0; i < N; ++i) c[i] = (i <= d) ? (S)b[i][k] : (S)0;
            int m = d;
#pragma unroll
            for (int lvl = 0; lvl < H; ++lvl) {
                if (m < 0) break;
                lo[lvl][k] = (float)c[0];
                hi[lvl][k] = (float)c[m < 0 ? 0 : m];
                if (m < 2) break;
                const S c0 = c[0], cm = c[m];
                const S mm = (S)m;
#pragma unroll
                for (int j = 0; j < N - 2; ++j) {
                    if (j <= m - 2) {
                        const S i1 = (S)(j + 1);
                        const S q = (c[j + 1] - c0) - (i1 / mm) * (cm - c0);
                        c[j] = q * (mm * (mm - (S)1)) / (i1 * (mm - (S)1 - (S)j));
                    }
                }
                m -= 2;
            }
        }
    }

    __device__ __forceinline__ void setup(const float (&b)[N][DIM], int deg)
    {
        d = Deg<D>::get(deg);
        if (d <= 5) setup_closed(b);
        else if (d >= kFp64Setup) setup_peel<double>(b);
        else setup_peel<float>(b);
    }

    __device__ __forceinline__ void eval(float t, float (&P)[DIM]) const
    {
        const float st = fmaf(-t, t, t);
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            if (D == 1 || (D == 0 && d == 1)) {
                P[k] = lerp(lo[0][k], hi[0][k], t);
                continue;
            }
            // innermost level kmax = floor(d/2): constant d_(d/2) for even d,
            // L(d_kmax, d_(d-kmax), t) for odd d
            float acc;
            const int kmax = (D ? D : d) / 2;
            if (D) {
                constexpr int KM = (D ? D : 2) / 2;
                acc = (D % 2 == 0) ? lo[KM][k] : lerp(lo[KM][k], hi[KM][k], t);
#pragma unroll
                for (int l = KM - 1; l >= 0; --l) acc = fmaf(st, acc, lerp(lo[l][k], hi[l][k], t));
            } else {
                acc = (d % 2 == 0) ? lo[kmax][k] : lerp(lo[kmax][k], hi[kmax][k], t);
                for (int l = kmax - 1; l >= 0; --l) acc = fmaf(st, acc, lerp(lo[l][k], hi[l][k], t));
            }
            P[k] = acc;
        }
    }
};


// ---------------------------------------------------------------- runtime degree

// Fallback for degrees not instantiated at compile time (and for dim != 3):
// the same arithmetic as the fixed-degree evaluators, written with plain
// loops over the runtime degree.  Setup is FP64 from degree 8 on.
template <int VAR, int DIM>
struct EvalDyn {
    static constexpr int N = kMaxDegree + 1;
    float c[N][DIM];          // Horner / centred: power coeffs; Bernstein: binom*b; dC: b
    float lo[N / 2 + 1][DIM]; // Seiler d_k
    float hi[N / 2 + 1][DIM]; // Seiler d_(d-k)
    int d;

    template <typename S>
    __device__ void setup_t(const float (&b)[N][DIM])
    {
        for (int k = 0; k < DIM; ++k) {
            S w[N];
            for (int i = 0; i <= d; ++i) w[i] = (S)b[i][k];
            if (VAR == VAR_HORNER) {
                for (int m = 1; m <= d; ++m)
                    for (int i = d; i >= m; --i) w[i] = w[i] - w[i - 1];
                S bin = 1;
                for (int i = 0; i <= d; ++i) {
                    c[i][k] = (float)(bin * w[i]);
                    bin = bin * (S)(d - i) / (S)(i + 1);
                }
            } else if (VAR == VAR_HORNER_CENTRED) {
                S bin = 1;
                for (int m = 0; m <= d; ++m) {
                    S h[N];
                    for (int i = 0; i <= d - m; ++i) h[i] = w[i];
                    for (int r = 1; r <= d - m; ++r)
                        for (int i = 0; i <= d - m - r; ++i) h[i] = (S)0.5 * (h[i] + h[i + 1]);
                    c[m][k] = (float)(bin * h[0]);
                    bin = bin * (S)(d - m) / (S)(m + 1);
                    for (int i = 0; i < d - m; ++i) w[i] = w[i + 1] - w[i];
                }
            } else if (VAR == VAR_SEILER) {
                int m = d;
                for (int lvl = 0; m >= 0; ++lvl) {
                    lo[lvl][k] = (float)w[0];
                    hi[lvl][k] = (float)w[m];
                    if (m < 2) break;
                    const S c0 = w[0], cm = w[m], mm = (S)m;
                    for (int j = 0; j <= m - 2; ++j) {
                        const S i1 = (S)(j + 1);
                        const S q = (w[j + 1] - c0) - (i1 / mm) * (cm - c0);
                        w[j] = q * (mm * (mm - (S)1)) / (i1 * (mm - (S)1 - (S)j));
                    }
                    m -= 2;
                }
            } else if (VAR == VAR_BERNSTEIN) {
                S bin = 1;
                for (int i = 0; i <= d; ++i) {
                    c[i][k] = (float)(bin * w[i]);
                    bin = bin * (S)(d - i) / (S)(i + 1);
                }
            } else {
                for (int i = 0; i <= d; ++i) c[i][k] = b[i][k];
            }
        }
    }
    __device__ void setup(const float (&b)[N][DIM], int deg)
    {
        d = deg;
        const int from = VAR == VAR_HORNER_CENTRED ? kFp64SetupCentred : kFp64Setup;
        if (d >= from && VAR != VAR_DECASTELJAU && VAR != VAR_BERNSTEIN) setup_t<double>(b);
        else setup_t<float>(b);
    }
    __device__ void eval(float t, float (&P)[DIM]) const
    {
        for (int k = 0; k < DIM; ++k) {
            float acc;
            if (VAR == VAR_HORNER || VAR == VAR_HORNER_CENTRED) {
                const float u = VAR == VAR_HORNER ? t : t - 0.5f;
                acc = c[d][k];
                for (int i = d - 1; i >= 0; --i) acc = fmaf(acc, u, c[i][k]);
            } else if (VAR == VAR_BERNSTEIN) {
                const float s = 1.0f - t;
                acc = 0.f;
                for (int i = 0; i <= d; ++i) {
                    float B = 1.f;
                    for (int r = 0; r < i; ++r) B *= t;
                    for (int r = 0; r < d - i; ++r) B *= s;
                    acc = fmaf(B, c[i][k], acc);
                }
            } else if (VAR == VAR_DECASTELJAU) {
                float w[N];
                for (int i = 0; i <= d; ++i) w[i] = c[i][k];
                for (int r = 1; r <= d; ++r)
                    for (int i = 0; i <= d - r; ++i) w[i] = lerp(w[i], w[i + 1], t);
                acc = w[0];
            } else {
                const float st = fmaf(-t, t, t);
                const int kmax = d / 2;
                if (d == 1) acc = lerp(lo[0][k], hi[0][k], t);
                else {
                    acc = (d % 2 == 0) ? lo[kmax][k] : lerp(lo[kmax][k], hi[kmax][k], t);
                    for (int l = kmax - 1; l >= 0; --l) acc = fmaf(st, acc, lerp(lo[l][k], hi[l][k], t));
                }
            }
            P[k] = acc;
        }
    }
};

template <int VAR, int D, int DIM>
struct Pick {
    using type = Eval<VAR, D, DIM>;
};
template <int VAR, int DIM>
struct Pick<VAR, 0, DIM> {
    using type = EvalDyn<VAR, DIM>;
};

// ---------------------------------------------------------------- kernel

constexpr int kWarps = 8;  // warps per block; one curve per warp per iteration
constexpr int kCurvesPerWarp = 8;  // curves per warp when the grid is not persistent
constexpr int kPairsPerWarp = 4;   // the same for the two-curves-per-warp kernel
constexpr int kGroupUnitsPerWarp = 2;  // and for the G-lanes-per-curve kernel
constexpr int kGroupWarps = 16;        // warps per block of the G-lanes-per-curve kernel (2 blocks per SM)
constexpr int kGroup8MinSamples = 128;  // samples per curve from which 8 lanes take a curve
constexpr int kGroup4MinSamples = 256;  // and from which 4 lanes do

template <int TM>
__device__ __forceinline__ float param(const CurveArgs& a, int64_t c, int j, uint32_t kc)
{
    if (TM == TM_ARRAY) return clamp01(__ldg(a.t + c * a.t_stride + j));
    if (TM == TM_UNIFORM) return a.n_t > 1 ? __fdiv_rn((float)j, (float)(a.n_t - 1)) : 0.f;
    if (TM == TM_HASH16) return hash_unit(lowbias32_premixed(kc, (uint32_t)j));
    return hash_unit(lowbias32(kc ^ (uint32_t)j));
}

// per-curve key of the in-kernel draw (pre-mixed for TM_HASH16)
template <int TM>
__device__ __forceinline__ uint32_t curve_key(const CurveArgs& a, int64_t c)
{
    if (TM != TM_HASH && TM != TM_HASH16) return 0u;
    const uint32_t kc = lowbias32(a.key ^ (uint32_t)(a.c_base + c));
    return TM == TM_HASH16 ? kc ^ (kc >> 16) : kc;
}

template <int DIM>
__device__ __forceinline__ float seg_len(const float (&p)[DIM], const float (&q)[DIM])
{
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const float e = p[k] - q[k];
        s = fmaf(e, e, s);
    }
    return sqrt_approx(s);
}

// Evaluate at the pre-mixed draw of sample index x = kg ^ i (TM_HASH16).  The
// centred form takes u = 1.m - 3/2 in one subtraction: 1.m - 1 and then - 1/2
// are both exact, so the value is the same as eval(t).
// `at` takes the draw's first product y = (km ^ j) * 0x7feb352d.
template <class E>
struct DrawEval {
    template <int DIM>
    __device__ __forceinline__ static void at(const E& e, uint32_t y, float (&P)[DIM])
    {
        e.eval(hash_one_plus(lowbias32_tail(y)) - 1.0f, P);
    }
};
template <int D, int DIM0>
struct DrawEval<Eval<VAR_HORNER_CENTRED, D, DIM0>> {
    template <int DIM>
    __device__ __forceinline__ static void at(const Eval<VAR_HORNER_CENTRED, D, DIM0>& e, uint32_t y,
                                              float (&P)[DIM])
    {
        e.eval_u(hash_one_plus(lowbias32_tail(y)) - 1.5f, P);
    }
};

// Polyline length over the samples [jb, je) of one lane with the pre-mixed
// draw.  jb is a multiple of 4, so sample jb + i (i < 4) has index
// (jb + i) == (g ^ i) for its group start g and km ^ (g ^ i) == (km ^ g) ^ i:
// one xor per sample gives the draw's input.  (Splitting the draw's first
// product into a per-group and a per-curve term saves that multiply but
// needs four more registers per lane, and measured slower.)  `first` and
// `last` return the run's end points for the join with the neighbouring
// lanes.
template <class E, int DIM, int UNROLL = 2>
__device__ __forceinline__ float run_length_h16(const E& e, uint32_t km, int jb, int je, float (&first)[DIM],
                                                float (&last)[DIM])
{
    float acc = 0.f;
    const uint32_t k0 = km ^ (uint32_t)jb;
    DrawEval<E>::at(e, k0 * kLowbiasMul1, first);
#pragma unroll
    for (int k = 0; k < DIM; ++k) last[k] = first[k];
#pragma unroll
    for (int i = 1; i < 4; ++i) {
        if (jb + i < je) {
            float P[DIM];
            DrawEval<E>::at(e, (k0 ^ (uint32_t)i) * kLowbiasMul1, P);
            acc += seg_len<DIM>(P, last);
#pragma unroll
            for (int k = 0; k < DIM; ++k) last[k] = P[k];
        }
    }
    int g = jb + 4;
#pragma unroll UNROLL
    for (; g + 4 <= je; g += 4) {
        // the group's 4 segments are summed first and then added to the run
        // (as many adds, rounding error growing with the run's groups)
        const uint32_t kg = km ^ (uint32_t)g;
        float gs = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float P[DIM];
            DrawEval<E>::at(e, (kg ^ (uint32_t)i) * kLowbiasMul1, P);
            const float sl = seg_len<DIM>(P, last);
            gs = i == 0 ? sl : gs + sl;
#pragma unroll
            for (int k = 0; k < DIM; ++k) last[k] = P[k];
        }
        acc += gs;
    }
    if (g < je) {
        const uint32_t kg = km ^ (uint32_t)g;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (g + i < je) {
                float P[DIM];
                DrawEval<E>::at(e, (kg ^ (uint32_t)i) * kLowbiasMul1, P);
                acc += seg_len<DIM>(P, last);
#pragma unroll
                for (int k = 0; k < DIM; ++k) last[k] = P[k];
            }
        }
    }
    return acc;
}

// Warp-per-curve kernel.  Warps are independent (no block barrier): each
// warp loads its curve's control points with one coalesced request (lane i
// reads element i), broadcasts them with shuffles, and prefetches the next
// curve's elements while it evaluates the current one.
template <int N, int DIM>
struct CtrlRegs {
    static constexpr int kPer = N * DIM;                  // elements per curve (upper bound)
    static constexpr int kLoads = (kPer + 31) / 32;       // elements per lane
    float v[kLoads];

    __device__ __forceinline__ void load(const CurveArgs& a, int64_t c, int per, int lane)
    {
#pragma unroll
        for (int r = 0; r < kLoads; ++r) {
            const int i = lane + 32 * r;
            v[r] = (c < a.n_curves && i < per) ? load_elem(a.ctrl, a.dtype, c * per + i) : 0.f;
        }
    }
    __device__ __forceinline__ void unpack(float (&b)[N][DIM], int deg) const
    {
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                const int e = i * DIM + k;
                const float x = __shfl_sync(kFull, v[e / 32], e % 32);
                b[i][k] = (i <= deg) ? x : 0.f;
            }
    }
};

template <int VAR, int D, int DIM, int TM, int OM>
__global__ void __launch_bounds__(kWarps * 32, 5) k_curve(const CurveArgs a)
{
    using E = typename Pick<VAR, D, DIM>::type;
    constexpr int N = E::N;
    __shared__ float s_stage[OM == OM_POINTS ? kWarps * 32 * DIM : 1];

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int deg = Deg<D>::get(a.degree);
    const int per = (deg + 1) * DIM;
    const int64_t n_warps = (int64_t)gridDim.x * kWarps;

    int64_t c = (int64_t)blockIdx.x * kWarps + wib;
    CtrlRegs<N, DIM> cur;
    cur.load(a, c, per, lane);
    for (; c < a.n_curves; c += n_warps) {
        E e;
        if constexpr (VAR == VAR_HORNER_CENTRED && D > 0 && DIM == 3) {
            e.setup_warp(cur.v[0], lane);
            cur.load(a, c + n_warps, per, lane);   // prefetch the next curve of this warp
        } else {
            float b[N][DIM];
            cur.unpack(b, deg);
            cur.load(a, c + n_warps, per, lane);
            e.setup(b, deg);
        }
        const uint32_t kc = curve_key<TM>(a, c);
        const int n_t = a.n_t;

        if (OM == OM_POINTS) {
            float* stage = s_stage + wib * 32 * DIM;
            for (int j0 = 0; j0 < n_t; j0 += 32) {
                const int j = j0 + lane;
                float P[DIM];
#pragma unroll
                for (int k = 0; k < DIM; ++k) P[k] = 0.f;
                if (j < n_t) e.eval(param<TM>(a, c, j, kc), P);
#pragma unroll
                for (int k = 0; k < DIM; ++k) stage[lane * DIM + k] = P[k];
                __syncwarp();
                const int valid = min(32, n_t - j0) * DIM;
                float* o = a.out + (c * n_t + j0) * DIM;
#pragma unroll
                for (int m = 0; m < DIM; ++m) {
                    const int idx = lane + 32 * m;
                    if (idx < valid) o[idx] = stage[idx];
                }
                __syncwarp();
            }
        } else {
            // each lane walks a contiguous run of samples; the segment
            // joining two runs is closed with one shuffle
            // (runs of a multiple of 4 samples under the pre-mixed draw)
            const int chunk = TM == TM_HASH16 ? (((n_t + 31) / 32 + 3) & ~3) : (n_t + 31) / 32;
            const int jb = lane * chunk;
            const int je = min(jb + chunk, n_t);
            float acc = 0.f;
            float first[DIM], prev[DIM];
#pragma unroll
            for (int k = 0; k < DIM; ++k) first[k] = prev[k] = 0.f;
            if (TM == TM_HASH16) {
                if (jb < je) acc = run_length_h16<E, DIM>(e, kc, jb, je, first, prev);
            } else if (jb < je) {
                e.eval(param<TM>(a, c, jb, kc), first);
#pragma unroll
                for (int k = 0; k < DIM; ++k) prev[k] = first[k];
#pragma unroll 4
                for (int j = jb + 1; j < je; ++j) {
                    float P[DIM];
                    e.eval(param<TM>(a, c, j, kc), P);
                    acc += seg_len<DIM>(P, prev);
#pragma unroll
                    for (int k = 0; k < DIM; ++k) prev[k] = P[k];
                }
            }
            float pl[DIM];
#pragma unroll
            for (int k = 0; k < DIM; ++k) pl[k] = __shfl_up_sync(kFull, prev[k], 1);
            if (lane > 0 && jb < je) acc += seg_len<DIM>(first, pl);
            acc = warp_sum(acc);
            if (lane == 0) a.out[c] = acc;
        }
    }
}

// Two curves per warp for the fused centred-Horner length of 3D curves of
// degree <= 4 under the pre-mixed draw: lanes 0-15 take curve 2 p, lanes
// 16-31 curve 2 p + 1.  Each half loads its 3 (d + 1) control values with
// one request, converts them cooperatively (setup_warp with a base lane),
// walks runs of a multiple of 4 samples per lane and reduces its length over
// 16 lanes, so the per-curve work (load, conversion, shuffles, reduction)
// is shared by twice the samples of a lane compared with one curve per warp.
// The sums run over 16 runs of about n_t / 16 samples.
template <int D>
__global__ void __launch_bounds__(kWarps * 32, 5) k_curve_pair(const CurveArgs a)
{
    using E = Eval<VAR_HORNER_CENTRED, D, 3>;
    constexpr int PER = 3 * (D + 1);
    static_assert(PER <= 16, "a half warp holds one curve's control values");
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int half = lane >> 4, li = lane & 15, base = lane & 16;
    const int64_t n_pairs = (a.n_curves + 1) / 2;
    const int64_t n_warps = (int64_t)gridDim.x * kWarps;
    auto load = [&](int64_t pr) {
        const int64_t c = 2 * pr + half;
        return (c < a.n_curves && li < PER) ? load_elem(a.ctrl, a.dtype, c * PER + li) : 0.f;
    };
    const int n_t = a.n_t;
    const int chunk = ((n_t + 15) / 16 + 3) & ~3;
    int64_t pr = (int64_t)blockIdx.x * kWarps + wib;
    float v = load(pr);
    for (; pr < n_pairs; pr += n_warps) {
        const int64_t c = 2 * pr + half;
        const bool live = c < a.n_curves;  // the last pair may have one curve
        E e;
        e.setup_warp(v, lane, base);
        v = load(pr + n_warps);  // prefetch this warp's next pair
        const uint32_t kc = curve_key<TM_HASH16>(a, c);
        const int jb = li * chunk;
        const int je = live ? min(jb + chunk, n_t) : jb;
        float acc = 0.f;
        float first[3] = {0.f, 0.f, 0.f}, prev[3] = {0.f, 0.f, 0.f};
        if (jb < je) acc = run_length_h16<E, 3>(e, kc, jb, je, first, prev);
        float pl[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) pl[k] = __shfl_up_sync(kFull, prev[k], 1);
        if (li > 0 && jb < je) acc += seg_len<3>(first, pl);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);  // within the half
        if (li == 0 && live) a.out[c] = acc;
    }
}

// G = 8 or 4 lanes per curve (4 or 8 curves per warp), for the same workload
// with more samples per curve: lanes G g .. G g + G - 1 take curve
// (32 / G) q + g.  Each group loads its 3 (d + 1) control values
// (ceil(3 (d + 1) / G) per lane), converts them redundantly (setup_group),
// walks runs of a multiple of 4 samples per lane and reduces its length over
// G lanes.  Against two curves per warp, a lane's per-curve work (load,
// conversion, key, run ends, reduction, store) is spread over 16 / G times
// the samples.  The sums run over G runs of about n_t / G samples.  (One or
// two lanes per curve measured slower at 1024 samples: 1.10e12 and 1.17e12
// against 1.18e12 points/s for 4.)  64 registers (4 blocks per SM) with the
// group loop unrolled by 4: 1.21e12 against 1.18e12 at 48 registers with 2;
// 80 registers measured slower.  Blocks of 16 warps (2 per SM) measured 1 %
// faster than 8 (4 per SM) or 4 (8 per SM).
template <int D, int G>
__global__ void __launch_bounds__(kGroupWarps * 32, 2) k_curve_group(const CurveArgs a)
{
    using E = Eval<VAR_HORNER_CENTRED, D, 3>;
    constexpr int PER = 3 * (D + 1);
    constexpr int NL = (PER + G - 1) / G;
    constexpr int CPW = 32 / G;  // curves per warp
    static_assert(G == 4 || G == 8, "4 or 8 lanes per curve");
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int grp = lane / G, li = lane % G, base = lane - li;
    const int64_t n_units = (a.n_curves + CPW - 1) / CPW;
    const int64_t n_warps = (int64_t)gridDim.x * kGroupWarps;
    float v[NL];
    auto load = [&](int64_t q) {
        const int64_t c = CPW * q + grp;
#pragma unroll
        for (int r = 0; r < NL; ++r) {
            const int i = li + G * r;
            v[r] = (c < a.n_curves && i < PER) ? load_elem(a.ctrl, a.dtype, c * PER + i) : 0.f;
        }
    };
    const int n_t = a.n_t;
    const int chunk = ((n_t + G - 1) / G + 3) & ~3;
    int64_t q = (int64_t)blockIdx.x * kGroupWarps + wib;
    load(q);
    for (; q < n_units; q += n_warps) {
        const int64_t c = CPW * q + grp;
        const bool live = c < a.n_curves;  // the warp's last unit may be partial
        E e;
        e.template setup_group<G>(v, base);
        load(q + n_warps);  // prefetch this warp's next curves
        const uint32_t kc = curve_key<TM_HASH16>(a, c);
        const int jb = li * chunk;
        const int je = live ? min(jb + chunk, n_t) : jb;
        float acc = 0.f;
        float first[3] = {0.f, 0.f, 0.f}, prev[3] = {0.f, 0.f, 0.f};
        if (jb < je) acc = run_length_h16<E, 3, 4>(e, kc, jb, je, first, prev);
        float pl[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) pl[k] = __shfl_up_sync(kFull, prev[k], 1);
        if (li > 0 && jb < je) acc += seg_len<3>(first, pl);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);  // within the group
        if (li == 0 && live) a.out[c] = acc;
    }
}

// ---------------------------------------------------------------- dispatch

// Grid of the pair kernel: as launch_one, with pairs of curves as the unit.
template <int D>
LaunchResult launch_pair(const CurveArgs& a, cudaStream_t s, const LaunchHooks& h)
{
    auto kern = k_curve_pair<D>;
    const int64_t n_pairs = (a.n_curves + 1) / 2;
    const int64_t work = (n_pairs + kWarps - 1) / kWarps;
    int grid = persistent_grid((const void*)kern, kWarps * 32, 0, h.sm_count, work);
    if (work > grid) {
        const int64_t g = (n_pairs + (int64_t)kWarps * kPairsPerWarp - 1) / ((int64_t)kWarps * kPairsPerWarp);
        if (g > grid) grid = (int)(g < 2147483647 ? g : 2147483647);
    }
    h.count(h.self);
    h.begin(h.self, s);
    kern<<<grid, kWarps * 32, 0, s>>>(a);
    cudaError_t err = cudaGetLastError();
    h.end(h.self, s);
    return {1, err};
}

// Grid of the G-lanes-per-curve kernel: units of 32 / G curves,
// kGroupUnitsPerWarp per warp when they outnumber the resident warps.
template <int D, int G>
LaunchResult launch_group(const CurveArgs& a, cudaStream_t s, const LaunchHooks& h)
{
    auto kern = k_curve_group<D, G>;
    const int64_t n_units = (a.n_curves + 32 / G - 1) / (32 / G);
    const int64_t work = (n_units + kGroupWarps - 1) / kGroupWarps;
    int grid = persistent_grid((const void*)kern, kGroupWarps * 32, 0, h.sm_count, work);
    if (work > grid) {
        const int64_t per = (int64_t)kGroupWarps * kGroupUnitsPerWarp;
        const int64_t g = (n_units + per - 1) / per;
        if (g > grid) grid = (int)(g < 2147483647 ? g : 2147483647);
    }
    h.count(h.self);
    h.begin(h.self, s);
    kern<<<grid, kGroupWarps * 32, 0, s>>>(a);
    cudaError_t err = cudaGetLastError();
    h.end(h.self, s);
    return {1, err};
}

template <int VAR, int D, int DIM, int TM, int OM>
LaunchResult launch_one(const CurveArgs& a, cudaStream_t s, const LaunchHooks& h)
{
    auto kern = k_curve<VAR, D, DIM, TM, OM>;
    const int64_t work = (a.n_curves + kWarps - 1) / kWarps;
    int grid = persistent_grid((const void*)kern, kWarps * 32, 0, h.sm_count, work);
    if (work > grid) {
        // More curves than resident warps: launch blocks of kCurvesPerWarp
        // curves per warp instead of a persistent grid.  The block scheduler
        // then refills SMs whose warps finish first.  With a persistent grid
        // every warp has a fixed share, warps progress unevenly, and 131,072
        // cubics averaged 32 of the 48 resident warps per SM.
        const int64_t g = (a.n_curves + (int64_t)kWarps * kCurvesPerWarp - 1) / ((int64_t)kWarps * kCurvesPerWarp);
        if (g > grid) grid = (int)(g < 2147483647 ? g : 2147483647);
    }
    h.count(h.self);
    h.begin(h.self, s);
    kern<<<grid, kWarps * 32, 0, s>>>(a);
    cudaError_t err = cudaGetLastError();
    h.end(h.self, s);
    return {1, err};
}

template <int VAR, int D, int DIM>
LaunchResult launch_modes(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h)
{
    if (om == OM_POINTS) {
        if (tm == TM_ARRAY) return launch_one<VAR, D, DIM, TM_ARRAY, OM_POINTS>(a, s, h);
        if (tm == TM_UNIFORM) return launch_one<VAR, D, DIM, TM_UNIFORM, OM_POINTS>(a, s, h);
        return launch_one<VAR, D, DIM, TM_HASH, OM_POINTS>(a, s, h);
    }
    if (tm == TM_ARRAY) return launch_one<VAR, D, DIM, TM_ARRAY, OM_LENGTH>(a, s, h);
    if (tm == TM_UNIFORM) return launch_one<VAR, D, DIM, TM_UNIFORM, OM_LENGTH>(a, s, h);
    // the fused evaluate-and-measure form of 3D curves of fixed degree gets the
    // pre-mixed draw when every sample index fits 16 bits; centred Horner up
    // to degree 4 runs two curves per warp from 64 samples, four from 128 and
    // eight from 256
    if constexpr (VAR == VAR_HORNER_CENTRED && D > 0 && D <= 4 && DIM == 3) {
        if (a.n_t >= kGroup4MinSamples && a.n_t <= 65536) return launch_group<D, 4>(a, s, h);
        if (a.n_t >= kGroup8MinSamples && a.n_t <= 65536) return launch_group<D, 8>(a, s, h);
        if (a.n_t >= 64 && a.n_t <= 65536) return launch_pair<D>(a, s, h);
    }
    if (D > 0 && DIM == 3 && a.n_t <= 65536) return launch_one<VAR, D, DIM, (D > 0 && DIM == 3 ? TM_HASH16 : TM_HASH), OM_LENGTH>(a, s, h);
    return launch_one<VAR, D, DIM, TM_HASH, OM_LENGTH>(a, s, h);
}

template <int VAR>
LaunchResult launch_curve_variant(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h)
{
    if (a.dim == 3) {
        switch (a.degree) {
        case 1: return launch_modes<VAR, 1, 3>(a, tm, om, s, h);
        case 2: return launch_modes<VAR, 2, 3>(a, tm, om, s, h);
        case 3: return launch_modes<VAR, 3, 3>(a, tm, om, s, h);
        case 4: return launch_modes<VAR, 4, 3>(a, tm, om, s, h);
        case 5: return launch_modes<VAR, 5, 3>(a, tm, om, s, h);
        case 6: return launch_modes<VAR, 6, 3>(a, tm, om, s, h);
        case 7: return launch_modes<VAR, 7, 3>(a, tm, om, s, h);
        default: return launch_modes<VAR, 0, 3>(a, tm, om, s, h);
        }
    }
    switch (a.dim) {
    case 1: return launch_modes<VAR, 0, 1>(a, tm, om, s, h);
    case 2: return launch_modes<VAR, 0, 2>(a, tm, om, s, h);
    default: return launch_modes<VAR, 0, 4>(a, tm, om, s, h);
    }
}

}  // namespace bez
