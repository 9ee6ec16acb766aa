// batch.cu -- mixed batches of Bezier curves, B-splines and NURBS evaluated by
// one persistent kernel (setup + evaluation captured in one CUDA graph).
//
// Every curve is a list of spans (a Bezier curve is one span).  The setup
// kernel (one thread per span component) forms each span of a spline by
// applying its extraction operator -- knot insertion done once per distinct
// (n_ctrl, degree) on the host in FP64 (spline.cuh span_operator) -- to the
// de Boor points, in homogeneous form for NURBS, in compensated FP32, and
// stores the span either as Bezier points (de Casteljau evaluation) or as
// power coefficients about tau = 1/2 (Horner evaluation), rounded once to
// FP32.
//
// Work is cut into items (a chunk of one curve's samples), each a 48-byte
// record holding everything its evaluation needs, sorted by class (degree,
// integral / rational).  The class evaluators run side by side on forked
// streams.  Warps take items round-robin, reading the next record while they
// evaluate the current item (static), or `grab` at a time from an atomic
// counter.  Within an item, each lane evaluates runs of 8 consecutive samples
// (1, 2 or 4 in a tile of at most 32, 64 or 128 samples)
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
constexpr int kItemsPerWarp = 4;  // static schedule: items per warp of a block

// ---------------------------------------------------------------- setup

// Component q of one span of degree P in its evaluation representation:
// Y = A X with A the span's operator -- its extraction operator M (splines;
// NURBS in homogeneous form), or T_p M / T_p for the power basis about 1/2
// (T_p, the Bezier -> centred map, is folded into the operators in FP64 on
// the host), or nothing for a Bezier curve in Bezier points.  Each operator
// entry is an unevaluated sum hi + lo of two floats (48 significant bits),
// each homogeneous point w P an exact sum (the product's error by one fma),
// and every row is a Dot2-style compensated dot product (Ogita, Rump & Oishi
// 2005): products split exactly by fma, partial sums by Knuth's TwoSum, the
// lower-order terms collected in a correction added once at the end.  The
// result is as accurate as a dot product in twice the working precision,
// then rounded once to FP32, at FP32 instruction rates (GB300 runs FP64 at a
// small fraction of FP32).
template <int P>
__device__ __forceinline__ void setup_comp(const BatchArgs& a, const SpanRec& r, int q, int comps)
{
    const bool spline = r.type != BEZ_CURVE_BEZIER;
    const bool rat = r.type == BEZ_CURVE_NURBS;
    const int dim = a.dim;
    const float* ctrl = a.ctrl_pool + r.ctrl;
    const float* wts = rat ? a.weight_pool + r.weight : nullptr;
    float xh[P + 1], xl[P + 1];  // X_j = xh_j + xl_j exactly
#pragma unroll
    for (int i = 0; i <= P; ++i) {
        if (rat) {
            const float w = __ldg(wts + i);
            if (q < dim) {
                const float v = __ldg(ctrl + (int64_t)i * dim + q);
                xh[i] = __fmul_rn(w, v);
                xl[i] = fmaf(w, v, -xh[i]);
            } else {
                xh[i] = w;
                xl[i] = 0.f;
            }
        } else {
            xh[i] = __ldg(ctrl + (int64_t)i * dim + q);
            xl[i] = 0.f;
        }
    }
    float* dst = a.span_pool + r.dst;
    if (!spline && a.repr == 0) {
#pragma unroll
        for (int i = 0; i <= P; ++i) dst[i * comps + q] = xh[i];
        return;
    }
    constexpr int S = kOpRowStride(P);
    const float2* M = a.op_pool + (spline ? r.op : a.tpow_off[P]);
    if (P <= 3 && !rat) {
        // Integral spans of degree <= 3: rows of at most 4 entries, so a plain
        // FP32 dot product (operator hi part by fma, lo parts summed apart)
        // stays within a few ulps of the row's absolute sum -- well inside
        // the evaluation's 1e-6 bar -- at a quarter of the compensated cost.
        // (Rational spans keep the compensated form: the plain one moved the
        // batch's NURBS error from 4.0e-7 to 5.7e-7 for 1 % of speed.)
#pragma unroll
        for (int i = 0; i <= P; ++i) {
            const float4* r4 = reinterpret_cast<const float4*>(M + i * S);
            float hi = 0.f, lo = 0.f;
#pragma unroll
            for (int q2 = 0; q2 < S / 2; ++q2) {
                const float4 v = __ldg(r4 + q2);
                if (2 * q2 <= P) {
                    hi = fmaf(v.x, xh[2 * q2], hi);
                    lo = fmaf(v.y, xh[2 * q2], lo);
                }
                if (2 * q2 + 1 <= P) {
                    hi = fmaf(v.z, xh[2 * q2 + 1], hi);
                    lo = fmaf(v.w, xh[2 * q2 + 1], lo);
                }
            }
            dst[i * comps + q] = hi + lo;
        }
        return;
    }
#pragma unroll
    for (int i = 0; i <= P; ++i) {
        float sh = 0.f, corr = 0.f;
        float2 row[S];
        const float4* r4 = reinterpret_cast<const float4*>(M + i * S);  // 16-byte aligned rows
#pragma unroll
        for (int q2 = 0; q2 < S / 2; ++q2) {
            const float4 v = __ldg(r4 + q2);
            row[2 * q2] = make_float2(v.x, v.y);
            row[2 * q2 + 1] = make_float2(v.z, v.w);
        }
#pragma unroll
        for (int j = 0; j <= P; ++j) {
            const float2 m = row[j];
            const float pr = __fmul_rn(m.x, xh[j]);
            float e = fmaf(m.x, xh[j], -pr);       // exact: m.x xh_j = pr + e
            e = fmaf(m.x, xl[j], e);               // lower-order terms
            e = fmaf(m.y, xh[j], e);
            const float t = __fadd_rn(sh, pr);     // TwoSum: sh + pr = t + err exactly
            const float bv = __fsub_rn(t, sh);
            const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bv)), __fsub_rn(pr, bv));
            sh = t;
            corr = __fadd_rn(corr, __fadd_rn(err, e));
        }
        dst[i * comps + q] = __fadd_rn(sh, corr);
    }
}

__device__ __forceinline__ SpanRec load_span_rec(const SpanRec* p)
{
    // three 16-byte loads, shared by the span's component threads through L1
    const int4* src = reinterpret_cast<const int4*>(p);
    const int4 x = __ldg(src), y = __ldg(src + 1), z = __ldg(src + 2);
    auto i64 = [](int lo, int hi) { return (int64_t)(((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo); };
    SpanRec r;
    r.ctrl = i64(x.x, x.y);
    r.weight = i64(x.z, x.w);
    r.dst = i64(y.x, y.y);
    r.op = i64(y.z, y.w);
    r.degree = z.x;
    r.type = z.y;
    r.reserved = 0;
    return r;
}

// Span extraction of span records [rec0, rec0 + n_rec), one thread per (span,
// component).  Each thread reads its span's record and then, independently
// of each other, the control points (and weights) and the operator rows.
// 48 registers (5 blocks of 256 per SM, 16 bytes of spill) rather than 62:
// the kernel waits on its operator and control-point loads, and the extra
// warps hide more of that than the spill costs (2 % of the batch launch)
__global__ void __launch_bounds__(256, 5) k_batch_setup(const BatchArgs a, int64_t rec0, int64_t n_rec)
{
    const int per = a.dim + 1;  // component slots per span (dim + 1 for homogeneous NURBS)
    const int64_t total = n_rec * per;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
        const int64_t sp = rec0 + idx / per;
        const int q = (int)(idx - (sp - rec0) * per);
        const SpanRec r = load_span_rec(a.span_rec + sp);
        const int comps = r.type == BEZ_CURVE_NURBS ? a.dim + 1 : a.dim;
        if (q >= comps) continue;
        switch (r.degree) {
        case 1: setup_comp<1>(a, r, q, comps); break;
        case 2: setup_comp<2>(a, r, q, comps); break;
        case 3: setup_comp<3>(a, r, q, comps); break;
        case 4: setup_comp<4>(a, r, q, comps); break;
        case 5: setup_comp<5>(a, r, q, comps); break;
        case 6: setup_comp<6>(a, r, q, comps); break;
        default: setup_comp<7>(a, r, q, comps); break;
        }
    }
}

// ---------------------------------------------------------------- evaluation

// Grid values t_j = fl32(j) / fl32(n - 1), the IEEE quotient.  For
// n - 1 < 2^16 without a division: q0 = RN(j r) with r = RN(1 / (n - 1)),
// then one correction step q0 + RN(j - q0 (n - 1)) r with both steps fused
// (Markstein's reciprocal-based division, 1990).  For every 0 <= j <= n - 1
// < 2^16 this equals the IEEE quotient (checked exhaustively, and the exact
// x = t of a degree-1 test curve is compared bit for bit on the GPU); larger
// grids divide.
struct GridDiv {
    float den, r;
    bool fast;
    __device__ __forceinline__ void init(int n)
    {
        den = (float)(n - 1);
        r = __frcp_rn((float)(n > 1 ? n - 1 : 1));
        fast = n > 1 && n - 1 < 65536;
    }
    __device__ __forceinline__ float operator()(int j) const
    {
        const float fj = (float)j;
        if (!fast) return den > 0.f ? __fdiv_rn(fj, den) : 0.f;
        const float q0 = __fmul_rn(fj, r);
        return fmaf(fmaf(-q0, den, fj), r, q0);
    }
};

// Span of t given the span s of an earlier, smaller parameter of the same
// run: the residual fma(t, ns, -s) is >= 0 with its exact sign, so s stands
// unless it reaches 1, when the full selection runs.  Same s and tau as
// uniform_span(t, ns, tau).
__device__ __forceinline__ int next_span(float t, int ns, int s, float& tau)
{
    const float r = fmaf(t, (float)ns, -(float)s);
    if (r >= 1.f && s < ns - 1) return uniform_span(t, ns, tau);
    tau = r;
    return s;
}

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
__device__ void item_fixed(const BatchArgs& a, const BatchItem& it, float* stage, int lane)
{
    constexpr bool RAT = C == 4;
    constexpr int DIM = 3;
    constexpr int LS = kRun * DIM + 1;  // padded per-lane stride of the tile
    const int n = it.n_samples;
    const bool spline = it.n_spans > 0;
    const int n_spans = it.n_spans;
    const int j0 = it.j0, j1 = it.j1;
    const float* base = a.span_pool + it.span_base;
    GridDiv grid;
    grid.init(n);
    float coef[P + 1][C];
    int cached = -1;
    float* out = a.out_pool + it.out_off;
    for (int tb = j0; tb < j1; tb += kTile) {
        // a tile of at most 32, 64 or 128 samples (a short item, the ragged
        // end of a long one) gives each lane a run of 1, 2 or 4 samples, so
        // the warp's lanes share it instead of a few lanes walking runs of 8
        const int vs = min(kTile, j1 - tb);
        const int lr = vs > 128 ? 3 : vs > 64 ? 2 : vs > 32 ? 1 : 0;  // log2 of the run
        const int my0 = tb + (lane << lr);
        int s_run = -1;  // span of this lane's previous sample in the run
#pragma unroll 2
        for (int r = 0; r < (1 << lr); ++r) {
            const int j = my0 + r;
            if (j < j1) {
                const float t = grid(j);
                float tau = t;
                int s = 0;
                if (spline) s = s_run < 0 ? uniform_span(t, n_spans, tau) : next_span(t, n_spans, s_run, tau);
                s_run = s;
                if (s != cached) {
                    // the span's (P + 1) C floats as whole float4s (16-byte aligned)
                    constexpr int S4 = kSpanStride(P, C) / 4;
                    const float4* src = reinterpret_cast<const float4*>(base + (int64_t)s * kSpanStride(P, C));
                    float v[4 * S4];
#pragma unroll
                    for (int m = 0; m < S4; ++m) {
                        const float4 x = __ldg(src + m);
                        v[4 * m] = x.x;
                        v[4 * m + 1] = x.y;
                        v[4 * m + 2] = x.z;
                        v[4 * m + 3] = x.w;
                    }
#pragma unroll
                    for (int i = 0; i <= P; ++i)
#pragma unroll
                        for (int q = 0; q < C; ++q) coef[i][q] = v[i * C + q];
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
        // Coalesced write-out: float f = 32 m + lane of the tile is element
        // f mod 24 of lane run f div 24 (a run is kRun * DIM = 24 floats).
        // With lane = 24 r0 + o0 and a = o0 div 8, run = r0 + m + w and
        // offset = o0 + 8 m - 24 w where w = (a + m) div 3, so its staged
        // position is base + m (LS + 8) + w (LS - 24).
        static_assert(kRun * DIM == 24 && LS == 25, "write-out index formula");
        const int valid = vs * DIM;
        if (lr == 3) {
            float* o = out + (int64_t)tb * DIM + lane;
            const int a3 = (lane % 24) / 8;
            const int base = (lane / 24) * LS + lane % 24;
#pragma unroll
            for (int m = 0; m < kRun * DIM; ++m) {
                const int w = m / 3 + ((m % 3) != 0 && a3 >= 3 - (m % 3) ? 1 : 0);
                if (32 * m + lane < valid) o[32 * m] = stage[base + m * (LS + 8) + w * (LS - 24)];
            }
        } else {
            // short runs: float f is component f mod 3 of sample f div 3,
            // element (sample mod run) of lane (sample div run)'s run
            float* o = out + (int64_t)tb * DIM;
            for (int f = lane; f < valid; f += 32) {
                const int smp = f / 3, q = f - 3 * smp;
                o[f] = stage[(smp >> lr) * LS + (smp & ((1 << lr) - 1)) * DIM + q];
            }
        }
        __syncwarp();
    }
}

// any dimension / degree (runtime loops)
template <int REPR>
__device__ void item_generic(const BatchArgs& a, const BatchItem& it, float* stage, int lane)
{
    const int dim = a.dim, p = it.degree;
    const bool spline = it.n_spans > 0, rat = it.rational != 0;
    const int n_spans = it.n_spans;
    const int j0 = it.j0, j1 = it.j1;
    const float* base = a.span_pool + it.span_base;
    const int comps = rat ? dim + 1 : dim;
    const int n = it.n_samples;
    const int LS = kRun * dim + 1;
    GridDiv grid;
    grid.init(n);
    float* out = a.out_pool + it.out_off;
    for (int tb = j0; tb < j1; tb += kTile) {
        const int my0 = tb + lane * kRun;
        int s_run = -1;
        for (int r = 0; r < kRun; ++r) {
            const int j = my0 + r;
            if (j >= j1) break;
            const float t = grid(j);
            float tau = t;
            int s = 0;
            if (spline) s = s_run < 0 ? uniform_span(t, n_spans, tau) : next_span(t, n_spans, s_run, tau);
            s_run = s;
            const float* src = base + (int64_t)s * kSpanStride(p, comps);
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

__device__ __forceinline__ BatchItem load_item(const BatchArgs& a, int64_t i)
{
    // every lane reads the same 48 bytes: three broadcast 16-byte loads
    const int4* src = reinterpret_cast<const int4*>(a.items + i);
    const int4 x = __ldg(src), y = __ldg(src + 1), z = __ldg(src + 2);
    BatchItem it;
    it.j0 = x.x;
    it.j1 = x.y;
    it.n_samples = x.z;
    it.n_spans = x.w;
    it.degree = y.x;
    it.rational = y.y;
    it.out_off = (int64_t)(((uint64_t)(uint32_t)y.w << 32) | (uint32_t)y.z);
    it.span_base = (int64_t)(((uint64_t)(uint32_t)z.y << 32) | (uint32_t)z.x);
    it.reserved = 0;
    return it;
}

// Evaluator of one item class: items [first, first + count) of the sorted
// table.  Static schedule: warp w takes items w, w + n_warps, ... and reads
// the record of its next item while it evaluates the current one; atomic
// schedule: `grab` items at a time from this class's counter.
template <int P, int C, int REPR>
__global__ void __launch_bounds__(256) k_batch_class(const BatchArgs a, int64_t first, int64_t count,
                                                     unsigned long long* counter)
{
    extern __shared__ float s_stage[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    float* stage = s_stage + wib * (32 * (kRun * a.dim + 1));
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    auto run = [&](const BatchItem& it) {
        if (P == 0) item_generic<REPR>(a, it, stage, lane);
        else item_fixed<(P > 0 ? P : 1), (C > 0 ? C : 3), REPR>(a, it, stage, lane);
    };
    if (a.schedule == 0) {
        int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
        if (item >= count) return;
        BatchItem nxt = load_item(a, first + item);
        for (; item < count; item += n_warps) {
            const BatchItem cur = nxt;
            if (item + n_warps < count) nxt = load_item(a, first + item + n_warps);
            run(cur);
        }
    } else {
        for (;;) {
            int64_t f = 0;
            if (lane == 0) f = (int64_t)atomicAdd(counter, (unsigned long long)a.grab);
            f = __shfl_sync(kFull, f, 0);
            if (f >= count) break;
            const int64_t last = min(f + a.grab, count);
            for (int64_t item = f; item < last; ++item) run(load_item(a, first + item));
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

static size_t batch_smem(const BatchArgs& a, int threads)
{
    return (size_t)(threads / 32) * 32 * (kRun * a.dim + 1) * sizeof(float);
}

int batch_full_grid(const BatchArgs& a, int threads, int sm_count, int cls)
{
    const void* kern = a.repr == 1 ? class_kernel<1>(cls) : class_kernel<0>(cls);
    const int64_t count = a.class_start[cls + 1] - a.class_start[cls];
    const int wpb = threads / 32;
    return persistent_grid(kern, threads, batch_smem(a, threads), sm_count, (count + wpb - 1) / wpb);
}

// span extraction of records [rec0, rec0 + n_rec) on stream s
static cudaError_t launch_setup(const BatchArgs& a, int64_t rec0, int64_t n_rec, int sm_count, cudaStream_t s,
                                const LaunchHooks& h, int* launches)
{
    if (n_rec <= 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>((n_rec * (a.dim + 1) + 255) / 256, (int64_t)sm_count * 16);
    h.count(h.self);
    k_batch_setup<<<grid > 0 ? grid : 1, 256, 0, s>>>(a, rec0, n_rec);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_batch(const BatchArgs& a, int threads, int sm_count, bool with_setup, cudaStream_t s,
                         const BatchStreams* bs, const LaunchHooks& h, int* launches)
{
    *launches = 0;
    cudaError_t e;
    int active = 0;
    for (int cls = 0; cls < kBatchClasses; ++cls) active += a.class_start[cls + 1] > a.class_start[cls];
    // class evaluators run side by side on forked streams; with the setup in
    // the same launch, each class's spans are extracted on its own stream just
    // before its evaluator, so one class's extraction overlaps the others'
    // evaluation
    const bool fork = bs && active > 1;
    const bool split_setup = with_setup && a.n_curves > 0 && fork;
    if (with_setup && a.n_curves > 0 && !split_setup) {
        if ((e = launch_setup(a, 0, a.n_span_rec, sm_count, s, h, launches)) != cudaSuccess) return e;
    }
    if (a.schedule != 0) {
        e = cudaMemsetAsync(a.counter, 0, kBatchClasses * sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
    }
    const size_t smem = batch_smem(a, threads);
    // Partitioned (atomic schedule): every class on a stream of its own with
    // a grid sized to its share of the measured work, so all classes are
    // resident together and finish at about the same time, each hiding the
    // others' latency; otherwise persistent grids on 4 shared streams.
    const bool part = a.partition != 0 && a.schedule != 0;
    const int nside = part ? kBatchSideStreams : kBatchSharedSideStreams;
    if (active == 0) return cudaSuccess;
    // fork the side streams off `s`
    h.begin(h.self, s);
    if (fork) {
        if ((e = cudaEventRecord(bs->fork, s)) != cudaSuccess) return e;
        for (int i = 0; i < nside; ++i)
            if ((e = cudaStreamWaitEvent(bs->side[i], bs->fork, 0)) != cudaSuccess) return e;
    }
    e = cudaSuccess;
    int m = 0;
    for (int cls = 0; cls < kBatchClasses && e == cudaSuccess; ++cls) {
        const int64_t first = a.class_start[cls], count = a.class_start[cls + 1] - first;
        const int64_t rec0 = a.span_class_start[cls], n_rec = a.span_class_start[cls + 1] - rec0;
        if (count <= 0 && !(split_setup && n_rec > 0)) continue;
        const int lane_of = fork ? m % (nside + 1) : 0;
        ++m;
        cudaStream_t cs = lane_of == 0 ? s : bs->side[lane_of - 1];
        if (split_setup && (e = launch_setup(a, rec0, n_rec, sm_count, cs, h, launches)) != cudaSuccess) break;
        if (count <= 0) continue;
        const void* kern = a.repr == 1 ? class_kernel<1>(cls) : class_kernel<0>(cls);
        const int wpb = threads / 32;
        int grid = persistent_grid(kern, threads, smem, sm_count, (count + wpb - 1) / wpb);
        if (part && a.class_grid[cls] > 0) grid = a.class_grid[cls];
        if (a.schedule == 0) {
            // blocks of kItemsPerWarp items per warp, scheduled by the hardware
            const int64_t g = (count + (int64_t)wpb * kItemsPerWarp - 1) / ((int64_t)wpb * kItemsPerWarp);
            if (g > grid) grid = (int)std::min<int64_t>(g, 2147483647);
        }
        unsigned long long* counter = static_cast<unsigned long long*>(a.counter) + cls;
        void* args[] = {(void*)&a, (void*)&first, (void*)&count, (void*)&counter};
        h.count(h.self);
        e = cudaLaunchKernel(kern, dim3(grid), dim3(threads), args, smem, cs);
        ++*launches;
    }
    if (fork) {
        // every side stream waited on the fork (and so joined a capture): join all of them back
        for (int i = 0; i < nside; ++i) {
            cudaError_t e2 = cudaEventRecord(bs->join[i], bs->side[i]);
            if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, bs->join[i], 0);
            if (e == cudaSuccess) e = e2;
        }
    }
    h.end(h.self, s);
    return e;
}

}  // namespace bez
