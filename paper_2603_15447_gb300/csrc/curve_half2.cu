// curve_half2.cu -- centred Horner in half2 arithmetic: the FP16-math
// evaluator (two samples per instruction), next to the FP16-storage /
// FP32-math forms of the other variants.
//
// Setup is the centred power basis of curve_eval.cuh (FP32, FP64 from degree
// 5), rounded once to half and broadcast to both halves of a half2.  A lane
// evaluates two samples at a time: u = t - 1/2 for both, packed into one
// half2, then d HFMA2 per coordinate.  Parameters come from the same draw,
// array or grid as the FP32 forms, and the polyline length is accumulated in
// FP32 from FP32 differences: squared segment lengths of densely sampled
// curves (~1e-5) sit below half's normal range.  Accuracy is that of 11-bit
// arithmetic on coefficients of magnitude up to ~2^d max|b| (about 1e-3 of
// the curve size for cubics); cubic 3D curves take 4.5 HFMA2 per point
// against 9 FFMA.
#include <cuda_fp16.h>

#include "curve_eval.cuh"

namespace bez {

template <int D>
struct EvalH2 {
    __half2 c[D + 1][3];  // centred power coefficients, both halves equal

    __device__ __forceinline__ void setup(const float (&b)[D + 1][3])
    {
        Eval<VAR_HORNER_CENTRED, D, 3> e;
        e.setup(b, D);
#pragma unroll
        for (int i = 0; i <= D; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) c[i][k] = __float2half2_rn(e.a[i][k]);
    }
    // samples at u = (u.lo, u.hi); P[k] holds coordinate k of both
    __device__ __forceinline__ void eval2(__half2 u, __half2 (&P)[3]) const
    {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            __half2 acc = c[D][k];
#pragma unroll
            for (int i = D - 1; i >= 0; --i) acc = __hfma2(acc, u, c[i][k]);
            P[k] = acc;
        }
    }
};

// samples j and j + 1 (j + 1 only if it exists: otherwise P1 repeats P0)
template <int D, int TM>
__device__ __forceinline__ void eval_pair(const EvalH2<D>& e, const CurveArgs& a, int64_t c, int j, uint32_t kc,
                                          float (&P0)[3], float (&P1)[3])
{
    const float t0 = param<TM>(a, c, j, kc);
    const float t1 = j + 1 < a.n_t ? param<TM>(a, c, j + 1, kc) : t0;
    __half2 P[3];
    e.eval2(__floats2half2_rn(t0 - 0.5f, t1 - 0.5f), P);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float2 f = __half22float2(P[k]);
        P0[k] = f.x;
        P1[k] = f.y;
    }
    if (TM == TM_ARRAY) {  // NaN parameters give NaN points
        if (t0 != t0) P0[0] = P0[1] = P0[2] = t0;
        if (t1 != t1) P1[0] = P1[1] = P1[2] = t1;
    }
}

template <int D, int TM, int OM>
__global__ void __launch_bounds__(kWarps * 32, 5) k_curve_h2(const CurveArgs a)
{
    constexpr int N = D + 1;
    __shared__ float s_stage[OM == OM_POINTS ? kWarps * 64 * 3 : 1];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t n_warps = (int64_t)gridDim.x * kWarps;
    int64_t c = (int64_t)blockIdx.x * kWarps + wib;
    CtrlRegs<N, 3> cur;
    cur.load(a, c, N * 3, lane);
    for (; c < a.n_curves; c += n_warps) {
        float b[N][3];
        cur.unpack(b, D);
        cur.load(a, c + n_warps, N * 3, lane);
        EvalH2<D> e;
        e.setup(b);
        const uint32_t kc = curve_key<TM>(a, c);
        const int n_t = a.n_t;
        if (OM == OM_POINTS) {
            // 64 samples per warp step: lane l takes samples 2l, 2l + 1
            float* stage = s_stage + wib * 64 * 3;
            for (int j0 = 0; j0 < n_t; j0 += 64) {
                const int j = j0 + 2 * lane;
                float P0[3] = {0.f, 0.f, 0.f}, P1[3] = {0.f, 0.f, 0.f};
                if (j < n_t) eval_pair<D, TM>(e, a, c, j, kc, P0, P1);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    stage[6 * lane + k] = P0[k];
                    stage[6 * lane + 3 + k] = P1[k];
                }
                __syncwarp();
                const int valid = min(64, n_t - j0) * 3;
                float* o = a.out + (c * n_t + j0) * 3;
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    const int idx = lane + 32 * m;
                    if (idx < valid) o[idx] = stage[idx];
                }
                __syncwarp();
            }
        } else {
            // runs of an even number of samples per lane, evaluated in pairs
            const int chunk = ((n_t + 31) / 32 + 1) & ~1;
            const int jb = lane * chunk;
            const int je = min(jb + chunk, n_t);
            float acc = 0.f;
            float first[3] = {0.f, 0.f, 0.f}, last[3] = {0.f, 0.f, 0.f};
            for (int j = jb; j < je; j += 2) {
                float P0[3], P1[3];
                eval_pair<D, TM>(e, a, c, j, kc, P0, P1);
                if (j == jb) {
#pragma unroll
                    for (int k = 0; k < 3; ++k) first[k] = P0[k];
                } else {
                    acc += seg_len<3>(P0, last);
                }
                if (j + 1 < je) {
                    acc += seg_len<3>(P1, P0);
#pragma unroll
                    for (int k = 0; k < 3; ++k) last[k] = P1[k];
                } else {
#pragma unroll
                    for (int k = 0; k < 3; ++k) last[k] = P0[k];
                }
            }
            float pl[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) pl[k] = __shfl_up_sync(kFull, last[k], 1);
            if (lane > 0 && jb < je) acc += seg_len<3>(first, pl);
            acc = warp_sum(acc);
            if (lane == 0) a.out[c] = acc;
        }
    }
}

template <int D>
static LaunchResult launch_h2(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h)
{
    const void* kern;
    if (om == OM_POINTS)
        kern = tm == TM_ARRAY     ? (const void*)k_curve_h2<D, TM_ARRAY, OM_POINTS>
               : tm == TM_UNIFORM ? (const void*)k_curve_h2<D, TM_UNIFORM, OM_POINTS>
                                  : (const void*)k_curve_h2<D, TM_HASH, OM_POINTS>;
    else
        kern = tm == TM_ARRAY     ? (const void*)k_curve_h2<D, TM_ARRAY, OM_LENGTH>
               : tm == TM_UNIFORM ? (const void*)k_curve_h2<D, TM_UNIFORM, OM_LENGTH>
                                  : (const void*)k_curve_h2<D, TM_HASH, OM_LENGTH>;
    const int64_t work = (a.n_curves + kWarps - 1) / kWarps;
    int grid = persistent_grid(kern, kWarps * 32, 0, h.sm_count, work);
    if (work > grid) {
        const int64_t g = (a.n_curves + (int64_t)kWarps * kCurvesPerWarp - 1) / ((int64_t)kWarps * kCurvesPerWarp);
        if (g > grid) grid = (int)(g < 2147483647 ? g : 2147483647);
    }
    void* args[] = {(void*)&a};
    h.count(h.self);
    h.begin(h.self, s);
    cudaError_t e = cudaLaunchKernel(kern, dim3(grid), dim3(kWarps * 32), args, 0, s);
    h.end(h.self, s);
    return {1, e};
}

LaunchResult launch_curve_half2(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h)
{
    switch (a.degree) {
    case 1: return launch_h2<1>(a, tm, om, s, h);
    case 2: return launch_h2<2>(a, tm, om, s, h);
    case 3: return launch_h2<3>(a, tm, om, s, h);
    case 4: return launch_h2<4>(a, tm, om, s, h);
    case 5: return launch_h2<5>(a, tm, om, s, h);
    case 6: return launch_h2<6>(a, tm, om, s, h);
    default: return launch_h2<7>(a, tm, om, s, h);
    }
}

}  // namespace bez
