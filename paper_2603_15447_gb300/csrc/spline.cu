// spline.cu -- B-spline and NURBS evaluation (paper Sec. 2.2): FP64 Boehm
// extraction of every span's Bezier control points, then FP32 de Casteljau
// on the span that holds each parameter.  See spline.cuh for the algorithm.
#include "curve_eval.cuh"
#include "spline.cuh"

namespace bez {

__global__ void k_spline_setup(const SplineArgs a)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.n_curves * a.n_spans) return;
    const int64_t c = idx / a.n_spans;
    const int s = (int)(idx % a.n_spans);
    const int n = a.n_ctrl, p = a.degree;
    const float* ctrl = a.ctrl + c * (int64_t)n * a.dim;
    const float* w = a.weights ? a.weights + c * (int64_t)n : nullptr;
    const float* U = a.knots ? a.knots + c * (int64_t)(n + p + 1) : nullptr;
    extract_span(ctrl, w, U, n, p, a.dim, s + p, a.spans + idx * (int64_t)(p + 1) * a.comps);
}

// parameter domain [lo, hi] = [U_p, U_n] of curve c
__device__ __forceinline__ void spline_domain(const SplineArgs& a, int64_t c, float& lo, float& hi)
{
    if (a.knots) {
        const float* U = a.knots + c * (int64_t)(a.n_ctrl + a.degree + 1);
        lo = __ldg(U + a.degree);
        hi = __ldg(U + a.n_ctrl);
    } else {
        lo = 0.f;
        hi = 1.f;
    }
}

template <int TM>
__device__ __forceinline__ float spline_param(const SplineArgs& a, int64_t c, int j, uint32_t kc, float lo, float hi)
{
    if (TM == TM_ARRAY) {
        const float t = __ldg(a.t + c * a.t_stride + j);
        return t < lo ? lo : (t > hi ? hi : t);
    }
    const float u = TM == TM_UNIFORM ? (a.n_t > 1 ? __fdiv_rn((float)j, (float)(a.n_t - 1)) : 0.f)
                                     : hash_unit(lowbias32(kc ^ (uint32_t)j));
    return a.knots ? fmaf(hi - lo, u, lo) : u;
}

// span index and local parameter of t
__device__ __forceinline__ int spline_span(const SplineArgs& a, int64_t c, float t, float& tau)
{
    const int ns = a.n_spans;
    if (!a.knots) {
        return uniform_span(t, ns, tau);
    }
    const float* B = a.knots + c * (int64_t)(a.n_ctrl + a.degree + 1) + a.degree;  // breakpoints B[0..ns]
    int lo = 0, hi = ns;  // count of B[i] <= t over i < ns, by bisection
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(B + mid) <= t) lo = mid + 1;
        else hi = mid;
    }
    int s = lo - 1;
    s = s < 0 ? 0 : s;
    const float b0 = __ldg(B + s), b1 = __ldg(B + s + 1);
    tau = (t - b0) / (b1 - b0);
    return s;
}

template <int P, int C, bool RAT>
__device__ __forceinline__ void spline_point(const SplineArgs& a, int64_t c, float t, float* out)
{
    float tau;
    const int s = spline_span(a, c, t, tau);
    const float* q = a.spans + ((c * a.n_spans + s) * (int64_t)(a.degree + 1)) * a.comps;
    if (P > 0) span_point_fixed<P, C, RAT>(q, tau, out);
    else span_point_dyn(q, a.degree, a.comps, a.weights != nullptr, tau, out);
    if (a.weights && out[a.comps - 1] == 0.f && a.err_word) atomicAdd(a.err_word, 1);
    if (t != t)
        for (int k = 0; k < a.comps; ++k) out[k] = t;
}

// one warp per curve; outputs as in the curve kernels
template <int P, int C, bool RAT, int TM, int OM>
__global__ void __launch_bounds__(kWarps * 32) k_spline(const SplineArgs a)
{
    __shared__ float s_stage[OM == OM_POINTS ? kWarps * 32 * 4 : 1];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int dim = a.dim;
    const int64_t n_warps = (int64_t)gridDim.x * kWarps;
    for (int64_t c = (int64_t)blockIdx.x * kWarps + wib; c < a.n_curves; c += n_warps) {
        float lo, hi;
        spline_domain(a, c, lo, hi);
        const uint32_t kc = (TM == TM_HASH) ? lowbias32(a.key ^ (uint32_t)c) : 0u;
        const int n_t = a.n_t;
        if (OM == OM_POINTS) {
            float* stage = s_stage + wib * 32 * 4;
            for (int j0 = 0; j0 < n_t; j0 += 32) {
                const int j = j0 + lane;
                float P_[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
                if (j < n_t) spline_point<P, C, RAT>(a, c, spline_param<TM>(a, c, j, kc, lo, hi), P_);
                for (int k = 0; k < dim; ++k) stage[lane * dim + k] = P_[k];
                __syncwarp();
                const int valid = min(32, n_t - j0) * dim;
                float* o = a.out + (c * n_t + j0) * dim;
                for (int idx = lane; idx < valid; idx += 32) o[idx] = stage[idx];
                __syncwarp();
            }
        } else {
            const int chunk = (n_t + 31) / 32;
            const int jb = lane * chunk;
            const int je = min(jb + chunk, n_t);
            float acc = 0.f;
            float first[4] = {0.f, 0.f, 0.f, 0.f}, prev[4] = {0.f, 0.f, 0.f, 0.f};
            for (int j = jb; j < je; ++j) {
                float P_[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
                spline_point<P, C, RAT>(a, c, spline_param<TM>(a, c, j, kc, lo, hi), P_);
                if (j == jb) {
                    for (int k = 0; k < 4; ++k) first[k] = P_[k];
                } else {
                    float s2 = 0.f;
                    for (int k = 0; k < dim; ++k) {
                        const float e = P_[k] - prev[k];
                        s2 = fmaf(e, e, s2);
                    }
                    acc += sqrt_approx(s2);
                }
                for (int k = 0; k < 4; ++k) prev[k] = P_[k];
            }
            float pl[4];
            for (int k = 0; k < 4; ++k) pl[k] = __shfl_up_sync(kFull, prev[k], 1);
            if (lane > 0 && jb < je) {
                float s2 = 0.f;
                for (int k = 0; k < dim; ++k) {
                    const float e = first[k] - pl[k];
                    s2 = fmaf(e, e, s2);
                }
                acc += sqrt_approx(s2);
            }
            acc = warp_sum(acc);
            if (lane == 0) a.out[c] = acc;
        }
    }
}

template <int P, int C, bool RAT>
static const void* pick_spline(int tm, int om)
{
    if (om == OM_POINTS)
        return tm == TM_ARRAY ? (const void*)k_spline<P, C, RAT, TM_ARRAY, OM_POINTS>
               : tm == TM_UNIFORM ? (const void*)k_spline<P, C, RAT, TM_UNIFORM, OM_POINTS>
                                  : (const void*)k_spline<P, C, RAT, TM_HASH, OM_POINTS>;
    return tm == TM_ARRAY ? (const void*)k_spline<P, C, RAT, TM_ARRAY, OM_LENGTH>
           : tm == TM_UNIFORM ? (const void*)k_spline<P, C, RAT, TM_UNIFORM, OM_LENGTH>
                              : (const void*)k_spline<P, C, RAT, TM_HASH, OM_LENGTH>;
}

LaunchResult launch_spline_setup(const SplineArgs& a, cudaStream_t s, const LaunchHooks& h)
{
    const int64_t n = a.n_curves * a.n_spans;
    if (n == 0) return {0, cudaSuccess};
    h.count(h.self);
    k_spline_setup<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(a);
    return {1, cudaGetLastError()};
}

LaunchResult launch_spline_eval(const SplineArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h)
{
    const bool rat = a.weights != nullptr;
    const void* kern;
    if (a.degree == 3 && a.dim == 3 && !rat) kern = pick_spline<3, 3, false>(tm, om);
    else if (a.degree == 3 && a.dim == 3 && rat) kern = pick_spline<3, 4, true>(tm, om);
    else kern = pick_spline<0, 0, false>(tm, om);
    const int grid = persistent_grid(kern, kWarps * 32, 0, h.sm_count, (a.n_curves + kWarps - 1) / kWarps);
    void* args[] = {(void*)&a};
    h.count(h.self);
    h.begin(h.self, s);
    cudaError_t e = cudaLaunchKernel(kern, dim3(grid), dim3(kWarps * 32), args, 0, s);
    h.end(h.self, s);
    return {1, e};
}

}  // namespace bez
