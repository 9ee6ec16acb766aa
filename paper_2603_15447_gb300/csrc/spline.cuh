// spline.cuh -- B-spline / NURBS support shared by the one-shot spline
// evaluators and the mixed-batch kernel.
//
// Setup (paper Sec. 2.2: "B-splines can be converted to piecewise Bezier
// curves using Boehm's algorithm"): every non-empty span [a, b) = [U_k,
// U_(k+1)) of a degree-p spline gets its own Bezier control points by knot
// insertion, in FP64, one thread per span.  Writing the de Boor points of the
// span as blossom values D_i = f(s_(i+1), ..., s_(i+p)) over the local knots
// s_1..s_2p = U_(k-p+1)..U_(k+p) (s_p = a, s_(p+1) = b):
//   left pass, levels l = 1..p-1, i = 0..p-l ascending:
//     Q_i <- lerp(Q_i, Q_(i+1), (a - s_(i+l)) / (s_(p+i+1) - s_(i+l)))
//   inserts a until every point carries a^(p-i); then
//   right pass, levels l = 1..p-1, i = p..l descending:
//     Q_i <- lerp(Q_(i-1), Q_i, (b - a) / (s_(p+i-l+1) - a))
//   inserts b, leaving Q_i = f(a^(p-i), b^i), the Bezier points of the span.
// Each step is one single-knot insertion restricted to the span's p+1 points
// (an affine combination of two blossom values that differ in one argument).
// Rational curves run the same steps on homogeneous points (w P, w).
//
// Evaluation: t is clamped to [U_p, U_n]; the span is the last non-empty one
// with U_k <= t (an interior knot starts the later span); tau = (t - a) /
// (b - a) (clamped uniform knots: see uniform_span);
// the span's Bezier points go through FP32 de Casteljau, and rational points
// are divided by their weight.
#pragma once

#include "common.cuh"

namespace bez {

// knot U_i of the clamped uniform vector: p+1 zeros, (i-p)/(n-p), p+1 ones
__host__ __device__ __forceinline__ double clamped_uniform_knot(int i, int n, int p)
{
    if (i <= p) return 0.0;
    if (i >= n) return 1.0;
    return (double)(i - p) / (double)(n - p);
}

// Knot-insertion passes on the p+1 de Boor points of one span, in place
// (rows of Q, `comps` columns), given the span's local knots s[1..2p].
// Returns false for an empty span (s_p == s_(p+1)), leaving Q untouched.
template <int MAXC>
__host__ __device__ inline bool boehm_span(double (&Q)[kMaxDegree + 1][MAXC], int comps, const double* s, int p)
{
    const double a = s[p], b = s[p + 1];
    if (!(a < b)) return false;
    for (int l = 1; l <= p - 1; ++l)
        for (int i = 0; i <= p - l; ++i) {
            const double lo = s[i + l], hi = s[p + i + 1];
            if (lo == a) continue;                 // weight 0: already a
            const double al = (a - lo) / (hi - lo);
            for (int q = 0; q < comps; ++q) Q[i][q] += al * (Q[i + 1][q] - Q[i][q]);
        }
    for (int l = 1; l <= p - 1; ++l)
        for (int i = p; i >= l; --i) {
            const double T = s[p + i - l + 1];
            if (T == b) continue;                  // weight 1: already b
            const double al = (b - a) / (T - a);
            for (int q = 0; q < comps; ++q) Q[i][q] = Q[i - 1][q] + al * (Q[i][q] - Q[i - 1][q]);
        }
    return true;
}

// local knots s[1..2p] = U_(k-p+1)..U_(k+p) of span k
__host__ __device__ inline void span_knots(const float* knots, int n, int p, int k, double* s)
{
    for (int j = 1; j <= 2 * p; ++j) {
        const int i = k - p + j;
        s[j] = knots ? (double)knots[i] : clamped_uniform_knot(i, n, p);
    }
}

// Bezier points of span k (p <= k < n) of one spline into q[(p+1)*comps]
// (FP32).  ctrl [n][dim], w [n] or NULL, knots [n+p+1] or NULL.
__device__ inline void extract_span(const float* ctrl, const float* w, const float* knots, int n, int p, int dim,
                                    int k, float* q_out)
{
    const int comps = w ? dim + 1 : dim;
    double s[2 * kMaxDegree + 1];   // s[1..2p]
    span_knots(knots, n, p, k, s);
    double Q[kMaxDegree + 1][5];
    for (int i = 0; i <= p; ++i) {
        const int g = k - p + i;
        const double wi = w ? (double)w[g] : 1.0;
        for (int q = 0; q < dim; ++q) Q[i][q] = wi * (double)ctrl[g * dim + q];
        if (w) Q[i][dim] = wi;
    }
    if (!boehm_span<5>(Q, comps, s, p)) {
        for (int i = 0; i <= p; ++i)
            for (int q = 0; q < comps; ++q) q_out[i * comps + q] = 0.f;
        return;
    }
    for (int i = 0; i <= p; ++i)
        for (int q = 0; q < comps; ++q) q_out[i * comps + q] = (float)Q[i][q];
}

// Extraction operator of span k of a degree-p spline with n control points:
// M[i][j] (row-major, (p+1)^2 doubles) maps the de Boor points
// P_(k-p+j) to the span's Bezier point i.  Knot insertion on unit vectors.
__host__ __device__ inline void span_operator(const float* knots, int n, int p, int k, double* M)
{
    double s[2 * kMaxDegree + 1];
    span_knots(knots, n, p, k, s);
    double Q[kMaxDegree + 1][kMaxDegree + 1];
    for (int i = 0; i <= p; ++i)
        for (int j = 0; j <= p; ++j) Q[i][j] = i == j ? 1.0 : 0.0;
    const bool nonempty = boehm_span<kMaxDegree + 1>(Q, p + 1, s, p);
    for (int i = 0; i <= p; ++i)
        for (int j = 0; j <= p; ++j) M[i * (p + 1) + j] = nonempty ? Q[i][j] : 0.0;
}

// Span of t on the clamped uniform knots k / ns: the largest k with
// t * ns >= k exactly.  fl(t * ns) can round across an integer when t lies
// within an ulp of a knot, which would evaluate the neighbouring span just
// outside its interval (a first-order error at the kinks of degree-1
// splines); the residual fma(t, ns, -k) has the exact sign of t * ns - k, so
// it corrects k, and the same residual is tau, rounded once.
__device__ __forceinline__ int uniform_span(float t, int ns, float& tau)
{
    const float fn = (float)ns;
    int s = (int)floorf(t * fn);
    s = s < 0 ? 0 : (s > ns - 1 ? ns - 1 : s);
    float r = fmaf(t, fn, -(float)s);
    if (r < 0.f && s > 0) {
        --s;
        r = fmaf(t, fn, -(float)s);
    } else if (r >= 1.f && s < ns - 1) {
        ++s;
        r = fmaf(t, fn, -(float)s);
    }
    tau = r;
    return s;
}

// FP32 de Casteljau on one span's Bezier points (compile-time degree P and
// component count C), rational division by the last component if RAT.
template <int P, int C, bool RAT>
__device__ __forceinline__ void span_point_fixed(const float* q, float tau, float* out)
{
#pragma unroll
    for (int c = 0; c < C; ++c) {
        float w[P + 1];
#pragma unroll
        for (int i = 0; i <= P; ++i) w[i] = q[i * C + c];
#pragma unroll
        for (int r = 1; r <= P; ++r)
#pragma unroll
            for (int i = 0; i <= P - r; ++i) w[i] = lerp(w[i], w[i + 1], tau);
        out[c] = w[0];
    }
    if (RAT) {
        const float inv = 1.0f / out[C - 1];
#pragma unroll
        for (int c = 0; c < C - 1; ++c) out[c] *= inv;
    }
}

// Runtime degree / component count (p <= kMaxDegree, comps <= 5).
__device__ inline void span_point_dyn(const float* q, int p, int comps, bool rat, float tau, float* out)
{
    for (int c = 0; c < comps; ++c) {
        float w[kMaxDegree + 1];
        for (int i = 0; i <= p; ++i) w[i] = q[i * comps + c];
        for (int r = 1; r <= p; ++r)
            for (int i = 0; i <= p - r; ++i) w[i] = lerp(w[i], w[i + 1], tau);
        out[c] = w[0];
    }
    if (rat) {
        const float inv = 1.0f / out[comps - 1];
        for (int c = 0; c < comps - 1; ++c) out[c] *= inv;
    }
}

}  // namespace bez
