// batch.cu -- mixed batches of Bezier curves, B-splines and NURBS evaluated by
// one persistent kernel (setup + evaluation captured in one CUDA graph).
//
// Work is cut into items (curve, chunk of `chunk` samples) listed in a table
// built on the host at plan creation.  Each warp of the persistent evaluator
// takes items either round-robin (static) or `grab` at a time from an atomic
// counter, reads the item's descriptor and evaluates its samples
// t_j = fl32(j) / fl32(n_samples - 1): Bezier curves by FP32 de Casteljau on
// their control points, B-splines / NURBS by de Casteljau on the Bezier span
// (extracted in FP64 by the setup kernel, spline.cuh) that holds t, rational
// points divided by their weight.  Points go out through a per-warp
// shared-memory transpose as coalesced stores.  Spline knots are the clamped
// uniform vectors.  chunk, schedule and block size are chosen by the
// autotuner in api.cu.
#include "curve_eval.cuh"
#include "spline.cuh"

namespace bez {

constexpr int kBatchMaxDeg = 7;

// de Casteljau for a compile-time degree on `comps` components read from q
// (q[i * comps + k]); rational results divided by the last component.
template <int P>
__device__ __forceinline__ void dc_fixed(const float* __restrict__ q, int comps, bool rat, float t, float* out)
{
    for (int k = 0; k < comps; ++k) {
        float w[P + 1];
#pragma unroll
        for (int i = 0; i <= P; ++i) w[i] = __ldg(q + i * comps + k);
#pragma unroll
        for (int r = 1; r <= P; ++r)
#pragma unroll
            for (int i = 0; i <= P - r; ++i) w[i] = lerp(w[i], w[i + 1], t);
        out[k] = w[0];
    }
    if (rat) {
        const float inv = 1.0f / out[comps - 1];
        for (int k = 0; k < comps - 1; ++k) out[k] *= inv;
    }
}

__device__ __forceinline__ void dc_any(const float* q, int p, int comps, bool rat, float t, float* out)
{
    switch (p) {
    case 1: dc_fixed<1>(q, comps, rat, t, out); break;
    case 2: dc_fixed<2>(q, comps, rat, t, out); break;
    case 3: dc_fixed<3>(q, comps, rat, t, out); break;
    case 4: dc_fixed<4>(q, comps, rat, t, out); break;
    case 5: dc_fixed<5>(q, comps, rat, t, out); break;
    case 6: dc_fixed<6>(q, comps, rat, t, out); break;
    default: dc_fixed<7>(q, comps, rat, t, out); break;
    }
}

// FP64 span extraction for the spline curves of the batch: one warp per
// spline curve, lanes over its spans.
__global__ void k_batch_setup(const BatchArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w; i < a.n_splines; i += n_warps) {
        const int64_t c = a.spline_ids[i];
        const bez_curve_desc dsc = a.desc[c];
        const int p = dsc.degree, n = dsc.n_ctrl;
        const bool rat = dsc.type == BEZ_CURVE_NURBS;
        const int comps = rat ? a.dim + 1 : a.dim;
        const float* ctrl = a.ctrl_pool + dsc.ctrl_off;
        const float* wts = rat ? a.weight_pool + dsc.weight_off : nullptr;
        for (int s = lane; s < n - p; s += 32)
            extract_span(ctrl, wts, nullptr, n, p, a.dim, s + p,
                         a.span_pool + a.span_off[c] + (int64_t)s * (p + 1) * comps);
    }
}

__device__ __forceinline__ void batch_item(const BatchArgs& a, int64_t item, float* stage, int lane)
{
    const int2 it = a.items[item];
    const int64_t c = it.x;
    const bez_curve_desc dsc = a.desc[c];
    const int n = dsc.n_samples;
    const int j0 = it.y * a.chunk;
    const int j1 = min(j0 + a.chunk, n);
    const int dim = a.dim;
    const int p = dsc.degree;
    const bool spline = dsc.type != BEZ_CURVE_BEZIER;
    const bool rat = dsc.type == BEZ_CURVE_NURBS;
    const int comps = rat ? dim + 1 : dim;
    const int n_spans = spline ? dsc.n_ctrl - p : 1;
    const float* base = spline ? a.span_pool + a.span_off[c] : a.ctrl_pool + dsc.ctrl_off;
    float* out = a.out_pool + dsc.out_off;
    const float den = (float)(n - 1);
    for (int jb = j0; jb < j1; jb += 32) {
        const int j = jb + lane;
        float P[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (j < j1) {
            const float t = n > 1 ? __fdiv_rn((float)j, den) : 0.f;
            if (spline) {
                float tau;
                const int s = uniform_span(t, n_spans, tau);
                dc_any(base + (int64_t)s * (p + 1) * comps, p, comps, rat, tau, P);
            } else {
                dc_any(base, p, dim, false, t, P);
            }
        }
        for (int k = 0; k < dim; ++k) stage[lane * dim + k] = P[k];
        __syncwarp();
        const int valid = min(32, j1 - jb) * dim;
        float* o = out + (int64_t)jb * dim;
        for (int idx = lane; idx < valid; idx += 32) o[idx] = stage[idx];
        __syncwarp();
    }
}

__global__ void k_batch_eval(const BatchArgs a)
{
    extern __shared__ float s_stage[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    float* stage = s_stage + wib * 32 * a.dim;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (a.schedule == 0) {
        for (int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; item < a.n_items; item += n_warps)
            batch_item(a, item, stage, lane);
    } else {
        for (;;) {
            int64_t first = 0;
            if (lane == 0) first = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(a.counter),
                                                      (unsigned long long)a.grab);
            first = __shfl_sync(kFull, first, 0);
            if (first >= a.n_items) break;
            const int64_t last = min(first + a.grab, a.n_items);
            for (int64_t item = first; item < last; ++item) batch_item(a, item, stage, lane);
        }
    }
}

cudaError_t launch_batch(const BatchArgs& a, int threads, int sm_count, bool with_setup, cudaStream_t s,
                         const LaunchHooks& h, int* launches)
{
    *launches = 0;
    cudaError_t e;
    if (with_setup && a.n_splines > 0) {
        const int64_t warps = a.n_splines;
        const int grid = (int)std::min<int64_t>((warps * 32 + 255) / 256, (int64_t)sm_count * 16);
        h.count(h.self);
        k_batch_setup<<<grid, 256, 0, s>>>(a);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (a.schedule != 0) {
        if ((e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    }
    const size_t smem = (size_t)threads / 32 * 32 * a.dim * sizeof(float);
    const int grid = persistent_grid((const void*)k_batch_eval, threads, smem, sm_count,
                                     (a.n_items + threads / 32 - 1) / (threads / 32));
    h.count(h.self);
    h.begin(h.self, s);
    k_batch_eval<<<grid, threads, smem, s>>>(a);
    e = cudaGetLastError();
    h.end(h.self, s);
    ++*launches;
    return e;
}

}  // namespace bez
