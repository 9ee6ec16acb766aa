/*
 * oracle.c -- plain FP64 CPU reference for batched Bezier / B-spline / NURBS /
 * tensor-product evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so and is
 * loaded only by tests/, by __graft_entry__.smoke() and by bench.py's CPU
 * baseline leg.  The product library never links, loads or calls it, and it
 * shares no code, header or table with the CUDA path.
 *
 * Every function computes the textbook definition of what the paper's method
 * reaches by a different route (texture filtering, de Casteljau, Seiler
 * interpolation, Horner), in double precision, with no blocking, fusion or
 * reordering:
 *   - Bezier curve: Bernstein sum  C(t) = sum_i binom(d,i) (1-t)^(d-i) t^i b_i
 *     (paper Sec. 2, the de Casteljau recursion it builds on, and Sec. 2.2 on
 *     the Bernstein basis).
 *   - Rational Bezier / NURBS: quotient of two integral curves, homogeneous
 *     weights (Sec. 2.2).
 *   - B-spline: Cox-de Boor recursion on a clamped knot vector (Sec. 2.2 names
 *     B-splines and Boehm knot insertion; the basis is the textbook one).
 *   - C0 piecewise chain: segment k = min(floor(t), N-1), local tau = t - k
 *     (Sec. 2.1 with Eq. 1-2; the oracle takes the logical control points).
 *   - Tensor-product surfaces and volumes: double / triple Bernstein sums
 *     (Sec. 2.2).
 *   - Gradients of the rational Bezier curve w.r.t. control points, weights
 *     and t (analytic derivatives of the quotient).
 *   - Polyline length sum_j |P_j - P_{j-1}| in index order.
 *   - lowbias32 counter hash (C. Wellons, "Prospecting for Hash Functions",
 *     2018), used only to reproduce parameters a kernel draws itself.
 *
 * Parameter handling (readings where the paper is silent):
 *   - t outside the domain is clamped to it; NaN propagates.
 *   - A tie at an integer t of a chain, or at an interior knot, goes to the
 *     later segment / span; t at the domain end goes to the last segment.
 *   - Uniform grids are t_a = fl32(a) / fl32(n-1) with IEEE single division
 *     (t_0 = 0 when n == 1), the same FP32 values a GPU kernel sees.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */

static double clamp_range(double t, double lo, double hi)
{
    if (t < lo) return lo;
    if (t > hi) return hi;
    return t; /* NaN falls through unchanged */
}

/* binomial coefficient; every partial product is itself a binomial, so the
 * divisions are exact for the small n used here */
static double binom(int n, int k)
{
    double r = 1.0;
    if (k < 0 || k > n) return 0.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

static double ipow(double x, int k)
{
    double r = 1.0;
    for (int i = 0; i < k; ++i) r *= x;
    return r;
}

/* Bernstein basis polynomial B_i^d(t) */
static double bernstein(int d, int i, double t)
{
    if (i < 0 || i > d) return 0.0;
    return binom(d, i) * ipow(1.0 - t, d - i) * ipow(t, i);
}

/* uniform grid value for index a of n: single-precision division */
double orc_grid_value(int64_t a, int64_t n)
{
    if (n <= 1) return 0.0;
    float num = (float)a;
    float den = (float)(n - 1);
    float q = num / den;
    return (double)q;
}

/* ------------------------------------------------------------------ */
/* Bezier curves (integral and rational)                               */
/* ------------------------------------------------------------------ */

/* One point of a (rational) Bezier curve of degree d at t (already clamped).
 * b: [d+1][dim]; w: [d+1] or NULL. */
static void bezier_point(const double* b, const double* w, int d, int dim, double t, double* out)
{
    double den = 0.0;
    for (int k = 0; k < dim; ++k) out[k] = 0.0;
    for (int i = 0; i <= d; ++i) {
        double B = bernstein(d, i, t);
        double wi = w ? w[i] : 1.0;
        for (int k = 0; k < dim; ++k) out[k] += B * wi * b[i * dim + k];
        den += B * wi;
    }
    if (w)
        for (int k = 0; k < dim; ++k) out[k] /= den;
}

/* ctrl [n_curves][d+1][dim]; weights [n_curves][d+1] or NULL;
 * t: element (c, j) at t[c * t_stride + j] (t_stride 0 = shared);
 * out [n_curves][n_t][dim]. */
void orc_bezier(const double* ctrl, const double* weights, int64_t n_curves, int degree, int dim,
                const double* t, int64_t t_stride, int64_t n_t, double* out)
{
    for (int64_t c = 0; c < n_curves; ++c) {
        const double* b = ctrl + c * (int64_t)(degree + 1) * dim;
        const double* w = weights ? weights + c * (int64_t)(degree + 1) : NULL;
        for (int64_t j = 0; j < n_t; ++j) {
            double tj = clamp_range(t[c * t_stride + j], 0.0, 1.0);
            bezier_point(b, w, degree, dim, tj, out + (c * n_t + j) * dim);
        }
    }
}

/* Same curves, parameter on the uniform grid a / (n_t - 1). */
void orc_bezier_grid(const double* ctrl, const double* weights, int64_t n_curves, int degree, int dim,
                     int64_t n_t, double* out)
{
    for (int64_t c = 0; c < n_curves; ++c) {
        const double* b = ctrl + c * (int64_t)(degree + 1) * dim;
        const double* w = weights ? weights + c * (int64_t)(degree + 1) : NULL;
        for (int64_t j = 0; j < n_t; ++j)
            bezier_point(b, w, degree, dim, orc_grid_value(j, n_t), out + (c * n_t + j) * dim);
    }
}

/* ------------------------------------------------------------------ */
/* C0 piecewise chains                                                 */
/* ------------------------------------------------------------------ */

/* ctrl [n_chains][n_seg*degree+1][dim] (logical control points, shared
 * endpoints); t in [0, n_seg]; out [n_chains][n_t][dim]. */
void orc_chain(const double* ctrl, int64_t n_chains, int n_seg, int degree, int dim,
               const double* t, int64_t t_stride, int64_t n_t, double* out)
{
    int64_t per_chain = (int64_t)n_seg * degree + 1;
    for (int64_t c = 0; c < n_chains; ++c) {
        for (int64_t j = 0; j < n_t; ++j) {
            double tj = clamp_range(t[c * t_stride + j], 0.0, (double)n_seg);
            double* o = out + (c * n_t + j) * dim;
            if (isnan(tj)) {
                for (int k = 0; k < dim; ++k) o[k] = tj;
                continue;
            }
            int64_t k = (int64_t)floor(tj);
            if (k > n_seg - 1) k = n_seg - 1;
            double tau = tj - (double)k;
            const double* b = ctrl + (c * per_chain + k * degree) * dim;
            bezier_point(b, NULL, degree, dim, tau, o);
        }
    }
}

/* ------------------------------------------------------------------ */
/* B-splines and NURBS (Cox-de Boor)                                    */
/* ------------------------------------------------------------------ */

/* clamped uniform knot vector: p+1 zeros, i/(n-p) for i = 1..n-p-1, p+1 ones */
void orc_clamped_uniform_knots(int n_ctrl, int degree, double* U)
{
    int m = n_ctrl + degree + 1;
    int n_int = n_ctrl - degree; /* number of spans */
    for (int i = 0; i < m; ++i) {
        if (i <= degree) U[i] = 0.0;
        else if (i >= n_ctrl) U[i] = 1.0;
        else U[i] = (double)(i - degree) / (double)n_int;
    }
}

/* span index k in [p, n-1] with U[k] <= u < U[k+1]; u == U[n] maps to the
 * last non-empty span */
static int find_span(const double* U, int n_ctrl, int p, double u)
{
    int k;
    for (k = n_ctrl - 1; k > p; --k)
        if (U[k] < U[k + 1] && U[k] <= u) break;
    return k;
}

/* All basis functions N_{i,p}(u), i = 0..n_ctrl-1, by the Cox-de Boor
 * triangle, 0/0 taken as 0.  N0 scratch must hold n_ctrl+p entries. */
static void cox_de_boor(const double* U, int n_ctrl, int p, double u, double* N)
{
    int m = n_ctrl + p; /* number of degree-0 functions */
    int span = find_span(U, n_ctrl, p, u);
    for (int i = 0; i < m; ++i) N[i] = (i == span) ? 1.0 : 0.0;
    for (int q = 1; q <= p; ++q) {
        for (int i = 0; i < m - q; ++i) {
            double left = 0.0, right = 0.0;
            double den1 = U[i + q] - U[i];
            double den2 = U[i + q + 1] - U[i + 1];
            if (den1 != 0.0) left = (u - U[i]) / den1 * N[i];
            if (den2 != 0.0) right = (U[i + q + 1] - u) / den2 * N[i + 1];
            N[i] = left + right;
        }
    }
}

/* ctrl [n_curves][n_ctrl][dim]; weights [n_curves][n_ctrl] or NULL
 * (integral B-spline); knots [n_curves][n_ctrl+degree+1] or NULL (clamped
 * uniform); t in knot space, clamped to [U[p], U[n]];
 * out [n_curves][n_t][dim]. */
void orc_bspline(const double* ctrl, const double* weights, const double* knots, int64_t n_curves,
                 int n_ctrl, int degree, int dim, const double* t, int64_t t_stride, int64_t n_t,
                 double* out)
{
    int m = n_ctrl + degree + 1;
    double* U = (double*)malloc(sizeof(double) * (size_t)m);
    double* N = (double*)malloc(sizeof(double) * (size_t)(n_ctrl + degree));
    for (int64_t c = 0; c < n_curves; ++c) {
        if (knots) for (int i = 0; i < m; ++i) U[i] = knots[c * m + i];
        else orc_clamped_uniform_knots(n_ctrl, degree, U);
        const double* P = ctrl + c * (int64_t)n_ctrl * dim;
        const double* w = weights ? weights + c * (int64_t)n_ctrl : NULL;
        for (int64_t j = 0; j < n_t; ++j) {
            double u = clamp_range(t[c * t_stride + j], U[degree], U[n_ctrl]);
            double* o = out + (c * n_t + j) * dim;
            if (isnan(u)) {
                for (int k = 0; k < dim; ++k) o[k] = u;
                continue;
            }
            cox_de_boor(U, n_ctrl, degree, u, N);
            double den = 0.0;
            for (int k = 0; k < dim; ++k) o[k] = 0.0;
            for (int i = 0; i < n_ctrl; ++i) {
                double wi = w ? w[i] : 1.0;
                for (int k = 0; k < dim; ++k) o[k] += N[i] * wi * P[i * dim + k];
                den += N[i] * wi;
            }
            if (w)
                for (int k = 0; k < dim; ++k) o[k] /= den;
        }
    }
    free(U);
    free(N);
}

/* ------------------------------------------------------------------ */
/* Tensor-product surfaces and volumes                                  */
/* ------------------------------------------------------------------ */

/* ctrl [n][du+1][dv+1][dim] -> out [n][nu][nv][dim], u_a, v_b on uniform grids */
void orc_surface(const double* ctrl, int64_t n, int du, int dv, int dim, int nu, int nv, double* out)
{
    for (int64_t s = 0; s < n; ++s) {
        const double* C = ctrl + s * (int64_t)(du + 1) * (dv + 1) * dim;
        for (int a = 0; a < nu; ++a) {
            double u = orc_grid_value(a, nu);
            for (int b = 0; b < nv; ++b) {
                double v = orc_grid_value(b, nv);
                double* o = out + (((s * nu) + a) * (int64_t)nv + b) * dim;
                for (int k = 0; k < dim; ++k) o[k] = 0.0;
                for (int i = 0; i <= du; ++i)
                    for (int j = 0; j <= dv; ++j) {
                        double B = bernstein(du, i, u) * bernstein(dv, j, v);
                        for (int k = 0; k < dim; ++k) o[k] += B * C[(i * (dv + 1) + j) * dim + k];
                    }
            }
        }
    }
}

/* ctrl [n][du+1][dv+1][dw+1][dim] -> out [n][nu][nv][nw][dim] */
void orc_volume(const double* ctrl, int64_t n, int du, int dv, int dw, int dim, int nu, int nv, int nw,
                double* out)
{
    int64_t per = (int64_t)(du + 1) * (dv + 1) * (dw + 1) * dim;
    for (int64_t s = 0; s < n; ++s) {
        const double* C = ctrl + s * per;
        for (int a = 0; a < nu; ++a) {
            double u = orc_grid_value(a, nu);
            for (int b = 0; b < nv; ++b) {
                double v = orc_grid_value(b, nv);
                for (int e = 0; e < nw; ++e) {
                    double w = orc_grid_value(e, nw);
                    double* o = out + ((((s * nu) + a) * (int64_t)nv + b) * nw + e) * dim;
                    for (int k = 0; k < dim; ++k) o[k] = 0.0;
                    for (int i = 0; i <= du; ++i)
                        for (int j = 0; j <= dv; ++j)
                            for (int l = 0; l <= dw; ++l) {
                                double B = bernstein(du, i, u) * bernstein(dv, j, v) * bernstein(dw, l, w);
                                const double* c = C + ((i * (dv + 1) + j) * (dw + 1) + l) * dim;
                                for (int k = 0; k < dim; ++k) o[k] += B * c[k];
                            }
                }
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Gradients of the (rational) Bezier curve                             */
/* ------------------------------------------------------------------ */

/* Given upstream gradient g [n_curves][n_t][dim] of a loss w.r.t. the curve
 * points C(t_j), accumulate
 *   grad_ctrl[c][i][k] = sum_j dC_j/dP_i . g_j      (w_i B_i / W)
 *   grad_w[c][i]       = sum_j B_i (P_i - C_j) . g_j / W_j
 *   grad_t (per-curve t: [c][j]; shared t: [j] summed over curves)
 *                      = g_j . (A'(t) - C W'(t)) / W   (zero where t was clamped)
 * where A = sum B_i w_i P_i and W = sum B_i w_i (w = 1 when weights == NULL).
 * Any output pointer may be NULL.  Outputs are overwritten. */
void orc_bezier_grad(const double* ctrl, const double* weights, int64_t n_curves, int degree, int dim,
                     const double* t, int64_t t_stride, int64_t n_t, const double* g,
                     double* grad_ctrl, double* grad_w, double* grad_t)
{
    int d = degree;
    if (grad_ctrl) for (int64_t i = 0; i < n_curves * (d + 1) * dim; ++i) grad_ctrl[i] = 0.0;
    if (grad_w) for (int64_t i = 0; i < n_curves * (d + 1); ++i) grad_w[i] = 0.0;
    if (grad_t) {
        int64_t len = t_stride ? n_curves * n_t : n_t;
        for (int64_t i = 0; i < len; ++i) grad_t[i] = 0.0;
    }
    double A[4], dA[4], C[4];
    for (int64_t c = 0; c < n_curves; ++c) {
        const double* P = ctrl + c * (int64_t)(d + 1) * dim;
        const double* w = weights ? weights + c * (int64_t)(d + 1) : NULL;
        for (int64_t j = 0; j < n_t; ++j) {
            double traw = t[c * t_stride + j];
            double tj = clamp_range(traw, 0.0, 1.0);
            const double* gj = g + (c * n_t + j) * dim;
            double W = 0.0, dW = 0.0;
            for (int k = 0; k < dim; ++k) { A[k] = 0.0; dA[k] = 0.0; }
            for (int i = 0; i <= d; ++i) {
                double B = bernstein(d, i, tj);
                double wi = w ? w[i] : 1.0;
                for (int k = 0; k < dim; ++k) A[k] += B * wi * P[i * dim + k];
                W += B * wi;
            }
            /* derivative via the hodograph: d * sum B_i^{d-1} (q_{i+1} - q_i) */
            for (int i = 0; i < d; ++i) {
                double B = bernstein(d - 1, i, tj);
                double w0 = w ? w[i] : 1.0, w1 = w ? w[i + 1] : 1.0;
                for (int k = 0; k < dim; ++k)
                    dA[k] += d * B * (w1 * P[(i + 1) * dim + k] - w0 * P[i * dim + k]);
                dW += d * B * (w1 - w0);
            }
            for (int k = 0; k < dim; ++k) C[k] = A[k] / W;
            for (int i = 0; i <= d; ++i) {
                double B = bernstein(d, i, tj);
                double wi = w ? w[i] : 1.0;
                if (grad_ctrl)
                    for (int k = 0; k < dim; ++k)
                        grad_ctrl[(c * (d + 1) + i) * dim + k] += B * wi / W * gj[k];
                if (grad_w) {
                    double dot = 0.0;
                    for (int k = 0; k < dim; ++k) dot += (P[i * dim + k] - C[k]) * gj[k];
                    grad_w[c * (d + 1) + i] += B * dot / W;
                }
            }
            if (grad_t) {
                double gt = 0.0;
                if (traw >= 0.0 && traw <= 1.0)
                    for (int k = 0; k < dim; ++k) gt += gj[k] * (dA[k] - C[k] * dW) / W;
                if (t_stride) grad_t[c * n_t + j] += gt;
                else grad_t[j] += gt;
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Polyline length                                                      */
/* ------------------------------------------------------------------ */

/* points [n][n_pts][dim] -> out[n] = sum_{j>=1} |P_j - P_{j-1}| */
void orc_polyline_length(const double* pts, int64_t n, int64_t n_pts, int dim, double* out)
{
    for (int64_t c = 0; c < n; ++c) {
        double L = 0.0;
        const double* p = pts + c * n_pts * dim;
        for (int64_t j = 1; j < n_pts; ++j) {
            double s = 0.0;
            for (int k = 0; k < dim; ++k) {
                double e = p[j * dim + k] - p[(j - 1) * dim + k];
                s += e * e;
            }
            L += sqrt(s);
        }
        out[c] = L;
    }
}

/* ------------------------------------------------------------------ */
/* Counter hash (to reproduce in-kernel parameter draws)                */
/* ------------------------------------------------------------------ */

/* Wellons' lowbias32: xorshift-multiply mixer with shifts 16, 15, 16 and
 * multipliers 0x7feb352d, 0x846ca68b. */
uint32_t orc_lowbias32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

/* Stream key for (seed, stream):
 *   key = h(lo(seed) ^ h(hi(seed) ^ h(stream))), h = lowbias32 */
uint32_t orc_stream_key(uint64_t seed, uint32_t stream)
{
    uint32_t lo = (uint32_t)(seed & 0xffffffffu), hi = (uint32_t)(seed >> 32);
    return orc_lowbias32(lo ^ orc_lowbias32(hi ^ orc_lowbias32(stream)));
}

/* Parameter draw j of curve c: u = (h >> 9) * 2^-23 with
 *   h = lowbias32(lowbias32(key ^ c) ^ j).
 * Writes t [n_curves][n_t] as doubles holding the exact FP32 values. */
void orc_hash_t(uint64_t seed, uint32_t stream, int64_t c0, int64_t n_curves, int64_t n_t, double* t)
{
    uint32_t key = orc_stream_key(seed, stream);
    for (int64_t c = 0; c < n_curves; ++c) {
        uint32_t kc = orc_lowbias32(key ^ (uint32_t)(c0 + c));
        for (int64_t j = 0; j < n_t; ++j) {
            uint32_t h = orc_lowbias32(kc ^ (uint32_t)j);
            t[c * n_t + j] = (double)(h >> 9) * (1.0 / 8388608.0);
        }
    }
}
