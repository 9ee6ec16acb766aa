// chain_eval.cuh -- C0 piecewise Bezier chains evaluated in registers.
//
// A chain of n_seg segments of degree p shares end points: segment k uses
// control points k*p .. k*p+p.  Global t in [0, n_seg] selects segment
// k = min(floor(t), n_seg-1) and local parameter tau = t - k (the reading
// used for ties: an integer t starts the later segment).  One warp owns a
// chain, stages its control points in shared memory, and evaluates each
// sample with the per-curve evaluators of curve_eval.cuh (setup per sample,
// since consecutive samples may fall in different segments).  Centred Horner
// on quadratic and cubic 3D chains stages the segments' power coefficients
// about tau = 1/2 instead (one conversion per segment, not per sample), one
// float4 per coefficient, so a sample reads d + 1 vectors and runs d FMA per
// coordinate.
#pragma once

#include "curve_eval.cuh"

namespace bez {

// global chain parameter of sample j, clamped to [0, n_seg] (NaN kept)
template <int TM>
__device__ __forceinline__ float chain_param(const CurveArgs& a, int64_t c, int j, uint32_t kc)
{
    const float ns = (float)a.n_seg;
    if (TM == TM_ARRAY) {
        const float t = __ldg(a.t + c * a.t_stride + j);
        return t < 0.f ? 0.f : (t > ns ? ns : t);
    }
    if (TM == TM_UNIFORM) return ns * (a.n_t > 1 ? __fdiv_rn((float)j, (float)(a.n_t - 1)) : 0.f);
    return ns * hash_unit(lowbias32(kc ^ (uint32_t)j));
}

__device__ __forceinline__ int chain_segment(float t, int n_seg)
{
    int k = (int)floorf(t);  // NaN converts to 0; the NaN then flows through tau
    k = k < 0 ? 0 : k;
    return k > n_seg - 1 ? n_seg - 1 : k;
}

// segments staged as centred power coefficients (float4 each)
template <int VAR, int D, int DIM>
__host__ __device__ constexpr bool chain_coef() { return VAR == VAR_HORNER_CENTRED && (D == 2 || D == 3) && DIM == 3; }

// shared floats per warp for the staged chain (control points or coefficients)
template <int VAR, int D, int DIM>
__host__ __device__ inline int chain_stage_floats(int n_seg, int degree)
{
    return chain_coef<VAR, D, DIM>() ? n_seg * (D + 1) * 4 : (n_seg * degree + 1) * DIM;
}

template <int VAR, int D, int DIM, int TM, int OM>
__global__ void __launch_bounds__(kWarps * 32) k_chain(const CurveArgs a)
{
    using E = typename Pick<VAR, D, DIM>::type;
    constexpr int N = E::N;
    constexpr bool COEF = chain_coef<VAR, D, DIM>();
    extern __shared__ float s_dyn[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int deg = Deg<D>::get(a.degree);
    const int n_pts = a.n_seg * deg + 1;
    const int per = n_pts * DIM;
    const int held = chain_stage_floats<VAR, D, DIM>(a.n_seg, deg);
    float* my = s_dyn + wib * held;
    float* stage = s_dyn + kWarps * held + wib * 32 * DIM;
    const int64_t n_warps = (int64_t)gridDim.x * kWarps;

    for (int64_t c = (int64_t)blockIdx.x * kWarps + wib; c < a.n_curves; c += n_warps) {
        if constexpr (COEF) {
            // lane per segment: its centred power coefficients a_m, m = 0..D
            float4* my4 = reinterpret_cast<float4*>(my);
            for (int sg = lane; sg < a.n_seg; sg += 32) {
                float b[N][DIM];
#pragma unroll
                for (int i = 0; i < N; ++i)
#pragma unroll
                    for (int q = 0; q < DIM; ++q) b[i][q] = load_elem(a.ctrl, a.dtype, c * per + (sg * D + i) * DIM + q);
                E e;
                e.setup(b, D);
#pragma unroll
                for (int m = 0; m < N; ++m) my4[sg * N + m] = make_float4(e.a[m][0], e.a[m][1], e.a[m][2], 0.f);
            }
        } else {
            for (int i = lane; i < per; i += 32) my[i] = load_elem(a.ctrl, a.dtype, c * per + i);
        }
        __syncwarp();
        const uint32_t kc = (TM == TM_HASH) ? lowbias32(a.key ^ (uint32_t)c) : 0u;
        const int n_t = a.n_t;
        auto point = [&](int j, float (&P)[DIM]) {
            const float t = chain_param<TM>(a, c, j, kc);
            const int k = chain_segment(t, a.n_seg);
            const float tau = t - (float)k;
            if constexpr (COEF) {
                const float4* sa = reinterpret_cast<const float4*>(my) + k * N;
                const float u = tau - 0.5f;
                float4 acc = sa[N - 1];
#pragma unroll
                for (int m = N - 2; m >= 0; --m) {
                    const float4 am = sa[m];
                    acc = make_float4(fmaf(acc.x, u, am.x), fmaf(acc.y, u, am.y), fmaf(acc.z, u, am.z), 0.f);
                }
                P[0] = acc.x;
                P[1] = acc.y;
                P[2] = acc.z;
            } else {
                float b[N][DIM];
                const float* src = my + k * deg * DIM;
#pragma unroll
                for (int i = 0; i < N; ++i)
#pragma unroll
                    for (int q = 0; q < DIM; ++q) b[i][q] = (i <= deg) ? src[i * DIM + q] : 0.f;
                E e;
                e.setup(b, deg);
                e.eval(tau, P);
            }
        };
        if (OM == OM_POINTS) {
            for (int j0 = 0; j0 < n_t; j0 += 32) {
                const int j = j0 + lane;
                float P[DIM];
#pragma unroll
                for (int q = 0; q < DIM; ++q) P[q] = 0.f;
                if (j < n_t) point(j, P);
#pragma unroll
                for (int q = 0; q < DIM; ++q) stage[lane * DIM + q] = P[q];
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
            const int chunk = (n_t + 31) / 32;
            const int jb = lane * chunk;
            const int je = min(jb + chunk, n_t);
            float acc = 0.f;
            float first[DIM], prev[DIM];
#pragma unroll
            for (int q = 0; q < DIM; ++q) first[q] = prev[q] = 0.f;
            if (jb < je) {
                point(jb, first);
#pragma unroll
                for (int q = 0; q < DIM; ++q) prev[q] = first[q];
                for (int j = jb + 1; j < je; ++j) {
                    float P[DIM];
                    point(j, P);
                    acc += seg_len<DIM>(P, prev);
#pragma unroll
                    for (int q = 0; q < DIM; ++q) prev[q] = P[q];
                }
            }
            float pl[DIM];
#pragma unroll
            for (int q = 0; q < DIM; ++q) pl[q] = __shfl_up_sync(kFull, prev[q], 1);
            if (lane > 0 && jb < je) acc += seg_len<DIM>(first, pl);
            acc = warp_sum(acc);
            if (lane == 0) a.out[c] = acc;
        }
        __syncwarp();  // every lane is done with `my` before the next chain overwrites it
    }
}

template <int VAR, int D, int DIM, int TM, int OM>
LaunchResult launch_chain_one(const CurveArgs& a, cudaStream_t s, const LaunchHooks& h)
{
    auto kern = k_chain<VAR, D, DIM, TM, OM>;
    const int held = chain_stage_floats<VAR, D, DIM>(a.n_seg, a.degree);
    const size_t smem = (size_t)kWarps * (held + 32 * DIM) * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return {0, e};
    }
    const int grid = persistent_grid((const void*)kern, kWarps * 32, smem, h.sm_count, (a.n_curves + kWarps - 1) / kWarps);
    h.count(h.self);
    h.begin(h.self, s);
    kern<<<grid, kWarps * 32, smem, s>>>(a);
    cudaError_t err = cudaGetLastError();
    h.end(h.self, s);
    return {1, err};
}

template <int VAR, int D, int DIM>
LaunchResult launch_chain_modes(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h)
{
    if (om == OM_POINTS) {
        if (tm == TM_ARRAY) return launch_chain_one<VAR, D, DIM, TM_ARRAY, OM_POINTS>(a, s, h);
        if (tm == TM_UNIFORM) return launch_chain_one<VAR, D, DIM, TM_UNIFORM, OM_POINTS>(a, s, h);
        return launch_chain_one<VAR, D, DIM, TM_HASH, OM_POINTS>(a, s, h);
    }
    if (tm == TM_ARRAY) return launch_chain_one<VAR, D, DIM, TM_ARRAY, OM_LENGTH>(a, s, h);
    if (tm == TM_UNIFORM) return launch_chain_one<VAR, D, DIM, TM_UNIFORM, OM_LENGTH>(a, s, h);
    return launch_chain_one<VAR, D, DIM, TM_HASH, OM_LENGTH>(a, s, h);
}

// quadratic and cubic 3D chains get fixed-degree kernels, the rest the
// runtime-degree evaluator
template <int VAR>
LaunchResult launch_chain_variant(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h)
{
    if (a.dim == 3 && a.degree == 2) return launch_chain_modes<VAR, 2, 3>(a, tm, om, s, h);
    if (a.dim == 3 && a.degree == 3) return launch_chain_modes<VAR, 3, 3>(a, tm, om, s, h);
    switch (a.dim) {
    case 1: return launch_chain_modes<VAR, 0, 1>(a, tm, om, s, h);
    case 2: return launch_chain_modes<VAR, 0, 2>(a, tm, om, s, h);
    case 3: return launch_chain_modes<VAR, 0, 3>(a, tm, om, s, h);
    default: return launch_chain_modes<VAR, 0, 4>(a, tm, om, s, h);
    }
}

}  // namespace bez
