// batch.cu -- mixed batches of Bezier curves, B-splines and NURBS evaluated by
// one persistent kernel (setup + evaluation captured in one CUDA graph).
//
// Every curve is a list of spans (a Bezier curve is one span).  The setup
// kernel (FP64, one warp per curve, lanes over spans) forms each span of a
// spline by applying its extraction operator -- knot insertion done once per
// distinct (n_ctrl, degree) on the host (spline.cuh span_operator) -- to the
// de Boor points, in homogeneous form for NURBS, and stores the span either
// as Bezier points (de Casteljau evaluation) or as power coefficients about
// tau = 1/2 (Horner evaluation), rounded once to FP32.
//
// Work is cut into items (curve, chunk of samples).  Warps take items
// round-robin (static) or `grab` at a time from an atomic counter.  Within an
// item, each lane evaluates runs of 8 consecutive samples
// t_j = fl32(j) / fl32(n_samples - 1), keeping the coefficients of its
// current span in registers and reloading them only when the span changes;
// results go through a padded per-warp shared-memory tile and out with
// coalesced stores.  Degree and component count are compile-time in the
// per-item dispatch for 3D curves.
#include "curve_eval.cuh"
#include "spline.cuh"

namespace bez {

constexpr int kRun = 8;              // consecutive samples per lane
constexpr int kTile = 32 * kRun;     // samples per warp sub-tile
constexpr int kBatchMaxComps = 5;

// ---------------------------------------------------------------- setup

// Bezier points b[0..p] (FP64) -> power coefficients about 1/2, in place:
// c_m = binom(p,m) * (Bernstein value at 1/2 of the m-th forward differences)
__device__ inline void bezier_to_centred(double* b, int p)
{
    double w[kMaxDegree + 1], c[kMaxDegree + 1];
    for (int i = 0; i <= p; ++i) w[i] = b[i];
    double bin = 1.0;
    for (int m = 0; m <= p; ++m) {
        double h[kMaxDegree + 1];
        for (int i = 0; i <= p - m; ++i) h[i] = w[i];
        for (int r = 1; r <= p - m; ++r)
            for (int i = 0; i <= p - m - r; ++i) h[i] = 0.5 * (h[i] + h[i + 1]);
        c[m] = bin * h[0];
        bin = bin * (double)(p - m) / (double)(m + 1);
        for (int i = 0; i < p - m; ++i) w[i] = w[i + 1] - w[i];
    }
    for (int i = 0; i <= p; ++i) b[i] = c[i];
}

__global__ void __launch_bounds__(256) k_batch_setup(const BatchArgs a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < a.n_span_tab; idx += stride) {
        const int2 cs = a.span_tab[idx];
        const int64_t c = cs.x;
        const int s = cs.y;
        const bez_curve_desc dsc = a.desc[c];
        const int p = dsc.degree;
        const bool spline = dsc.type != BEZ_CURVE_BEZIER;
        const bool rat = dsc.type == BEZ_CURVE_NURBS;
        const int dim = a.dim;
        const int comps = rat ? dim + 1 : dim;
        const float* ctrl = a.ctrl_pool + dsc.ctrl_off;
        const float* wts = rat ? a.weight_pool + dsc.weight_off : nullptr;
        {
            const double* M = spline ? a.op_pool + a.span_ops[a.op_off[c] + s] : nullptr;
            float* dst = a.span_pool + a.span_off[c] + (int64_t)s * (p + 1) * comps;
            for (int q = 0; q < comps; ++q) {
                double P[kMaxDegree + 1], Q[kMaxDegree + 1];
                for (int i = 0; i <= p; ++i) {
                    const int g = s + i;
                    const double wi = rat ? (double)__ldg(wts + g) : 1.0;
                    P[i] = q < dim ? wi * (double)__ldg(ctrl + (int64_t)g * dim + q) : wi;
                }
                for (int i = 0; i <= p; ++i) {
                    if (!spline) {
                        Q[i] = P[i];
                        continue;
                    }
                    double acc = 0.0;
                    for (int j = 0; j <= p; ++j) acc = fma(M[i * (p + 1) + j], P[j], acc);
                    Q[i] = acc;
                }
                if (a.repr == 1) bezier_to_centred(Q, p);
                for (int i = 0; i <= p; ++i) dst[i * comps + q] = (float)Q[i];
            }
        }
    }
}

// ---------------------------------------------------------------- evaluation

template <int P, int C, int REPR>
__device__ __forceinline__ void span_eval(const float (&k)[P + 1][C], float tau, float (&out)[C])
{
    if (REPR == 1) {
        const float u = tau - 0.5f;
#pragma unroll
        for (int q = 0; q < C; ++q) {
            float acc = k[P][q];
#pragma unroll
            for (int i = P - 1; i >= 0; --i) acc = fmaf(acc, u, k[i][q]);
            out[q] = acc;
        }
    } else {
#pragma unroll
        for (int q = 0; q < C; ++q) {
            float w[P + 1];
#pragma unroll
            for (int i = 0; i <= P; ++i) w[i] = k[i][q];
#pragma unroll
            for (int r = 1; r <= P; ++r)
#pragma unroll
                for (int i = 0; i <= P - r; ++i) w[i] = lerp(w[i], w[i + 1], tau);
            out[q] = w[0];
        }
    }
}

// one item of a 3D curve with compile-time degree P; C = 3 (integral) or 4
// (rational, homogeneous)
template <int P, int C, int REPR>
__device__ void item_fixed(const BatchArgs& a, const bez_curve_desc& dsc, const float* base, int n_spans, int j0,
                           int j1, float* stage, int lane)
{
    constexpr bool RAT = C == 4;
    constexpr int DIM = 3;
    constexpr int LS = kRun * DIM + 1;  // padded per-lane stride of the tile
    const int n = dsc.n_samples;
    const bool spline = dsc.type != BEZ_CURVE_BEZIER;
    const float den = (float)(n - 1);
    float coef[P + 1][C];
    int cached = -1;
    float* out = a.out_pool + dsc.out_off;
    for (int tb = j0; tb < j1; tb += kTile) {
        const int my0 = tb + lane * kRun;
#pragma unroll 2
        for (int r = 0; r < kRun; ++r) {
            const int j = my0 + r;
            if (j < j1) {
                const float t = n > 1 ? __fdiv_rn((float)j, den) : 0.f;
                float tau = t;
                const int s = spline ? uniform_span(t, n_spans, tau) : 0;
                if (s != cached) {
                    const float* src = base + (int64_t)s * (P + 1) * C;
#pragma unroll
                    for (int i = 0; i <= P; ++i)
#pragma unroll
                        for (int q = 0; q < C; ++q) coef[i][q] = __ldg(src + i * C + q);
                    cached = s;
                }
                float pt[C];
                span_eval<P, C, REPR>(coef, tau, pt);
                if (RAT) {
                    const float inv = 1.0f / pt[C - 1];
#pragma unroll
                    for (int q = 0; q < DIM; ++q) pt[q] *= inv;
                }
#pragma unroll
                for (int q = 0; q < DIM; ++q) stage[lane * LS + r * DIM + q] = pt[q];
            }
        }
        __syncwarp();
        const int valid = min(kTile, j1 - tb) * DIM;
        float* o = out + (int64_t)tb * DIM;
        for (int idx = lane; idx < valid; idx += 32) {
            const int smp = idx / DIM, q = idx - smp * DIM;
            o[idx] = stage[(smp / kRun) * LS + (smp % kRun) * DIM + q];
        }
        __syncwarp();
    }
}

// any dimension / degree (runtime loops)
template <int REPR>
__device__ void item_generic(const BatchArgs& a, const bez_curve_desc& dsc, const float* base, int n_spans, int j0,
                             int j1, float* stage, int lane)
{
    const int dim = a.dim, p = dsc.degree;
    const bool spline = dsc.type != BEZ_CURVE_BEZIER, rat = dsc.type == BEZ_CURVE_NURBS;
    const int comps = rat ? dim + 1 : dim;
    const int n = dsc.n_samples;
    const int LS = kRun * dim + 1;
    const float den = (float)(n - 1);
    float* out = a.out_pool + dsc.out_off;
    for (int tb = j0; tb < j1; tb += kTile) {
        const int my0 = tb + lane * kRun;
        for (int r = 0; r < kRun; ++r) {
            const int j = my0 + r;
            if (j >= j1) break;
            const float t = n > 1 ? __fdiv_rn((float)j, den) : 0.f;
            float tau = t;
            const int s = spline ? uniform_span(t, n_spans, tau) : 0;
            const float* src = base + (int64_t)s * (p + 1) * comps;
            float pt[kBatchMaxComps];
            for (int q = 0; q < comps; ++q) {
                float w[kMaxDegree + 1];
                for (int i = 0; i <= p; ++i) w[i] = __ldg(src + i * comps + q);
                if (REPR == 1) {
                    const float u = tau - 0.5f;
                    float acc = w[p];
                    for (int i = p - 1; i >= 0; --i) acc = fmaf(acc, u, w[i]);
                    pt[q] = acc;
                } else {
                    for (int rr = 1; rr <= p; ++rr)
                        for (int i = 0; i <= p - rr; ++i) w[i] = lerp(w[i], w[i + 1], tau);
                    pt[q] = w[0];
                }
            }
            if (rat) {
                const float inv = 1.0f / pt[comps - 1];
                for (int q = 0; q < dim; ++q) pt[q] *= inv;
            }
            for (int q = 0; q < dim; ++q) stage[lane * LS + r * dim + q] = pt[q];
        }
        __syncwarp();
        const int valid = min(kTile, j1 - tb) * dim;
        float* o = out + (int64_t)tb * dim;
        for (int idx = lane; idx < valid; idx += 32) {
            const int smp = idx / dim, q = idx - smp * dim;
            o[idx] = stage[(smp / kRun) * LS + (smp % kRun) * dim + q];
        }
        __syncwarp();
    }
}

// Item classes: 3D curves get one kernel per (degree, integral / rational),
// everything else the generic kernel; the host sorts items by class.
int batch_item_class(const bez_curve_desc& d, int dim)
{
    if (dim != 3) return kBatchClasses - 1;
    return (d.type == BEZ_CURVE_NURBS ? 7 : 0) + (d.degree - 1);
}

__device__ __forceinline__ void item_range(const BatchArgs& a, int64_t item, const bez_curve_desc*& dsc_out,
                                           bez_curve_desc& dsc, int& j0, int& j1, int& n_spans, const float*& base)
{
    const int2 it = a.items[item];
    const int64_t c = it.x;
    dsc = a.desc[c];
    j0 = it.y * a.chunk;
    j1 = min(j0 + a.chunk, dsc.n_samples);
    n_spans = dsc.type != BEZ_CURVE_BEZIER ? dsc.n_ctrl - dsc.degree : 1;
    base = a.span_pool + a.span_off[c];
    dsc_out = &dsc;
}

// Persistent evaluator of one item class: items [first, first + count) of the
// sorted table, taken round-robin or from this class's atomic counter.
template <int P, int C, int REPR>
__global__ void __launch_bounds__(256) k_batch_class(const BatchArgs a, int64_t first, int64_t count,
                                                     unsigned long long* counter)
{
    extern __shared__ float s_stage[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    float* stage = s_stage + wib * (32 * (kRun * a.dim + 1));
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    auto run = [&](int64_t item) {
        bez_curve_desc dsc;
        const bez_curve_desc* dp;
        int j0, j1, n_spans;
        const float* base;
        item_range(a, first + item, dp, dsc, j0, j1, n_spans, base);
        if (P == 0) item_generic<REPR>(a, dsc, base, n_spans, j0, j1, stage, lane);
        else item_fixed<(P > 0 ? P : 1), (C > 0 ? C : 3), REPR>(a, dsc, base, n_spans, j0, j1, stage, lane);
    };
    if (a.schedule == 0) {
        for (int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; item < count; item += n_warps) run(item);
    } else {
        for (;;) {
            int64_t f = 0;
            if (lane == 0) f = (int64_t)atomicAdd(counter, (unsigned long long)a.grab);
            f = __shfl_sync(kFull, f, 0);
            if (f >= count) break;
            const int64_t last = min(f + a.grab, count);
            for (int64_t item = f; item < last; ++item) run(item);
        }
    }
}

template <int REPR>
static const void* class_kernel(int cls)
{
    switch (cls) {
    case 0: return (const void*)k_batch_class<1, 3, REPR>;
    case 1: return (const void*)k_batch_class<2, 3, REPR>;
    case 2: return (const void*)k_batch_class<3, 3, REPR>;
    case 3: return (const void*)k_batch_class<4, 3, REPR>;
    case 4: return (const void*)k_batch_class<5, 3, REPR>;
    case 5: return (const void*)k_batch_class<6, 3, REPR>;
    case 6: return (const void*)k_batch_class<7, 3, REPR>;
    case 7: return (const void*)k_batch_class<1, 4, REPR>;
    case 8: return (const void*)k_batch_class<2, 4, REPR>;
    case 9: return (const void*)k_batch_class<3, 4, REPR>;
    case 10: return (const void*)k_batch_class<4, 4, REPR>;
    case 11: return (const void*)k_batch_class<5, 4, REPR>;
    case 12: return (const void*)k_batch_class<6, 4, REPR>;
    case 13: return (const void*)k_batch_class<7, 4, REPR>;
    default: return (const void*)k_batch_class<0, 0, REPR>;
    }
}

cudaError_t launch_batch(const BatchArgs& a, int threads, int sm_count, bool with_setup, cudaStream_t s,
                         const LaunchHooks& h, int* launches)
{
    *launches = 0;
    cudaError_t e;
    if (with_setup && a.n_curves > 0) {
        const int grid = (int)std::min<int64_t>((a.n_span_tab + 255) / 256, (int64_t)sm_count * 16);
        h.count(h.self);
        k_batch_setup<<<grid > 0 ? grid : 1, 256, 0, s>>>(a);
        ++*launches;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (a.schedule != 0) {
        e = cudaMemsetAsync(a.counter, 0, kBatchClasses * sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
    }
    const size_t smem = (size_t)(threads / 32) * 32 * (kRun * a.dim + 1) * sizeof(float);
    bool first_kernel = true;
    e = cudaSuccess;
    for (int cls = 0; cls < kBatchClasses; ++cls) {
        const int64_t first = a.class_start[cls], count = a.class_start[cls + 1] - first;
        if (count <= 0) continue;
        const void* kern = a.repr == 1 ? class_kernel<1>(cls) : class_kernel<0>(cls);
        const int grid = persistent_grid(kern, threads, smem, sm_count, (count + threads / 32 - 1) / (threads / 32));
        unsigned long long* counter = static_cast<unsigned long long*>(a.counter) + cls;
        void* args[] = {(void*)&a, (void*)&first, (void*)&count, (void*)&counter};
        h.count(h.self);
        if (first_kernel) h.begin(h.self, s);
        first_kernel = false;
        e = cudaLaunchKernel(kern, dim3(grid), dim3(threads), args, smem, s);
        ++*launches;
        if (e != cudaSuccess) break;
    }
    if (!first_kernel) h.end(h.self, s);
    return e;
}

}  // namespace bez
