// internal.h -- declarations shared between the libbez host runtime and the
// kernel translation units.  Not part of the public ABI (see include/bez.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bez.h"

namespace bez {

// Arguments of the register curve evaluators (one warp per curve).
struct CurveArgs {
    const void* ctrl;   // [n_curves][degree+1][dim], element type `dtype`
    int32_t dtype;      // 0 f32, 1 f16, 2 bf16
    int32_t degree;
    int32_t dim;
    int32_t n_t;
    int64_t n_curves;
    const float* t;     // TM_ARRAY: t[c * t_stride + j]
    int64_t t_stride;
    float* out;         // OM_POINTS [n_curves][n_t][dim]; OM_LENGTH [n_curves]
    uint32_t key;       // TM_HASH stream key
    int32_t n_seg;      // chains: segments per chain (0 for single curves)
    int64_t c_base;     // global index of curve 0 of this launch (the draw hashes c_base + c)
};

// Result of a launcher: how many kernels it launched and the CUDA status.
struct LaunchResult {
    int launches;
    cudaError_t err;
};

// Hooks the runtime passes to launchers so that the main kernel of a call is
// bracketed by timing events and counted.
struct LaunchHooks {
    void (*count)(void* self);                  // every kernel launch
    void (*begin)(void* self, cudaStream_t s);  // main kernel of a call
    void (*end)(void* self, cudaStream_t s);
    void* self;
    int sm_count;
};

// Register evaluators, one translation unit per variant (curve_<var>.cu).
LaunchResult launch_curve_horner(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h);
LaunchResult launch_curve_horner_centred(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h);
LaunchResult launch_curve_bernstein(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h);
LaunchResult launch_curve_decasteljau(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h);
LaunchResult launch_curve_seiler(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h);
// centred Horner in half2 arithmetic (dim 3, degree 1..7)
LaunchResult launch_curve_half2(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h);

// ---------------------------------------------------------------- textures

// A cudaArray-backed atlas with a linear-filtering texture object for reads
// and a surface object for the packers' writes.  fmt 0: float4 texels,
// fmt 1: half4 texels.  depth 0 means a 2D array.
struct Atlas {
    cudaArray_t arr = nullptr;
    cudaTextureObject_t tex = 0;
    cudaSurfaceObject_t surf = 0;
    int w = 0, h = 0, depth = 0, fmt = 0;
};
cudaError_t atlas_ensure(Atlas& at, int w, int h, int depth, int fmt);
void atlas_free(Atlas& at);

// Texture state owned by a context.
struct TexState {
    Atlas dc3;    // 3D de Casteljau tiles / strips: texel(x,y,z) = b_(x+y+z)
    Atlas strip2; // 2D strips: texel(x,y) = b_(x+y)
    Atlas seil2;  // 2D 2x2 Seiler tiles (degree 2, 3)
    Atlas seil2s; // 2D (s+1) x (s+1) spread Seiler tiles (degree 2, 3)
    Atlas seil3;  // 3D 2x2x2 Seiler tiles (degree 4, 5)
    Atlas chain;  // zig-zag C0 chain textures
    Atlas chain3; // cubic zig-zag chain textures, (N+1) x 2 x 2 per chain
    Atlas probe;  // 2x2x2 weight probe
    Atlas probe2; // 2x2 weight probe (one-hot texels)
    Atlas surf3;  // bicubic surface tiles: four column cubics per 2x2x2 RGBA tile
    Atlas surf2;  // bicubic surface tiles in the 2x2 Seiler layout, one column cubic per channel
    float4* rescale = nullptr;  // unorm tiles: per tile (offset, scale)
    int64_t rescale_cap = 0;    // tiles the rescale buffer holds
    int max3d = 16384, max2d_w = 131072, max2d_h = 65536;
};

// Texel storage format of an atlas (TEXEL_* of texel.cuh) for an input
// dtype and a bez_tex_format; the rescale buffer of unorm atlases, n tiles.
int texel_format(int dtype, int tex_format);
cudaError_t rescale_buffer(TexState& ts, int fmt, int64_t n, float4** out);

// Texture evaluators: pack the control points into the atlas of `variant`,
// then evaluate.  `variant` is a bez_variant texture value.
// `spread` > 1 selects the spread Seiler tile (TEX_SEILER, degree 2, 3).
LaunchResult launch_tex_curve(const CurveArgs& a, int variant, int tm, int om, int tex_format, int spread,
                              TexState& ts, cudaStream_t s, const LaunchHooks& h);
// Co-issue: `share` of every 8 samples through the tex2D Seiler tile, the
// rest by centred Horner (cubic, dim 3, hashed t with n_t <= 65536, length).
constexpr int kDefaultTexShare = 2;
LaunchResult launch_tex_coissue(const CurveArgs& a, int share, int tex_format, TexState& ts, cudaStream_t s,
                                const LaunchHooks& h);
// 2D probe: out[i] = the four bilinear texel weights at coords xy[i].
LaunchResult launch_tex_probe2d(const float* xy, int64_t n, float* out, TexState& ts, cudaStream_t s,
                                const LaunchHooks& h);
// Filter-weight probe: out[i] = filtered (x, y, z) texel index at coords xyz[i].
LaunchResult launch_tex_probe(const float* xyz, int64_t n, float* out, TexState& ts, cudaStream_t s,
                              const LaunchHooks& h);

// C0 chains (chain_*.cu): register evaluators per segment.
LaunchResult launch_chain_horner(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h);
LaunchResult launch_chain_horner_centred(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h);
LaunchResult launch_chain_bernstein(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h);
LaunchResult launch_chain_decasteljau(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h);
LaunchResult launch_chain_seiler(const CurveArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h);
// Zig-zag texture for C0 quadratic chains (tex.cu).
// `spread` s >= 1: each 2x2 window sampled on an (s+1) x (s+1) texel grid.
LaunchResult launch_tex_chain(const CurveArgs& a, int tm, int om, int spread, int tex_format, TexState& ts, cudaStream_t s,
                              const LaunchHooks& h);
constexpr int kChainMaxFloats = 3072;  // (n_seg*degree+1)*dim per chain staged in shared memory

// ---------------------------------------------------------------- splines

struct SplineArgs {
    const float* ctrl;     // [n_curves][n_ctrl][dim]
    const float* weights;  // [n_curves][n_ctrl] or NULL (integral B-spline)
    const float* knots;    // [n_curves][n_ctrl+degree+1] or NULL (clamped uniform)
    int64_t n_curves;
    int32_t n_ctrl, degree, dim;
    int32_t comps;         // dim, or dim+1 for homogeneous rational points
    int32_t n_spans;       // n_ctrl - degree
    float* spans;          // scratch [n_curves][n_spans][degree+1][comps]
    const float* t;
    int64_t t_stride;
    int32_t n_t;
    float* out;
    uint32_t key;
    int32_t* err_word;
};
LaunchResult launch_spline_setup(const SplineArgs& a, cudaStream_t s, const LaunchHooks& h);
LaunchResult launch_spline_eval(const SplineArgs& a, int tm, int om, cudaStream_t s, const LaunchHooks& h);

// ---------------------------------------------------------------- surfaces / volumes

struct TensorArgs;
struct TensorLaunch {
    const void* ctrl;
    int32_t dtype;
    int64_t n;
    int32_t du, dv, dw;  // dw < 0: surface
    int32_t dim;
    int32_t nu, nv, nw;
    float* out;
};
LaunchResult launch_tensor_product(const TensorLaunch& t, cudaStream_t s, const LaunchHooks& h);
// Bicubic surfaces (nu <= kSurfTexMaxRows) and tricubic scalar volumes (nu <=
// kVolTexMaxRows, nw a multiple of 4, out 16-byte aligned) through RGBA
// texture tiles, texels in the storage format of `tex_format` (a
// bez_tex_format).
constexpr int kSurfTexMaxRows = 64;
constexpr int kVolTexMaxRows = 32;
LaunchResult launch_tex_surface(const TensorLaunch& t, bool seiler, int tex_format, int spread, TexState& ts,
                                cudaStream_t s, const LaunchHooks& h);
size_t tensor_product_smem(const TensorLaunch& t);

// ---------------------------------------------------------------- adjoint

struct GradArgs {
    const float* ctrl;     // [n][d+1][dim]
    const float* weights;  // [n][d+1] or NULL
    int64_t n_curves;
    int32_t degree, dim, n_t;
    const float* t;        // t[c * t_stride + j]
    int64_t t_stride;
    const float* g;        // [n][n_t][dim]
    float* grad_ctrl;      // [n][d+1][dim] or NULL
    float* grad_w;         // [n][d+1] or NULL
    float* grad_t;         // [n][n_t] (per-curve t) or [n_t] (shared t) or NULL
    int32_t shared_gt;     // shared-t sums staged in shared memory (n_t small enough)
    const float* target;   // fused squared error: [n][n_t][dim] targets (g is then formed in-kernel), or NULL
    float loss_scale;      // loss = loss_scale * sum ||C - target||^2, g = 2 loss_scale (C - target)
    float* loss;           // [n] per-curve loss (fused form) or NULL
};

LaunchResult launch_grad(const GradArgs& a, cudaStream_t s, const LaunchHooks& h);

// ---------------------------------------------------------------- mixed batches

// One work item of a batch: a chunk of one curve's samples with everything
// the evaluator needs, so a warp reads one record (prefetched) per item.
struct alignas(16) BatchItem {
    int32_t j0, j1;     // samples [j0, j1) of the curve
    int32_t n_samples;  // the curve's sample count
    int32_t n_spans;    // spline spans; 0 for a Bezier curve (no span selection)
    int32_t degree;
    int32_t rational;
    int64_t out_off;    // floats into out_pool: the curve's first point
    int64_t span_base;  // floats into span_pool: the curve's first span
    int64_t reserved;
};
static_assert(sizeof(BatchItem) == 48, "BatchItem is read as three 16-byte loads");

// Side streams of a batch: class evaluators run concurrently between a fork
// and a join on the launching stream (also inside graph capture).
constexpr int kBatchSideStreams = 14;  // one stream per class when the GPU is partitioned between them
constexpr int kBatchSharedSideStreams = 3;  // otherwise classes share the main stream and 3 side streams
struct BatchStreams {
    cudaStream_t side[kBatchSideStreams];
    cudaEvent_t fork;
    cudaEvent_t join[kBatchSideStreams];
};

// One span of a batch as the setup kernel reads it, with every offset
// resolved on the host so that its loads depend on this record alone.
struct alignas(16) SpanRec {
    int64_t ctrl;    // floats into ctrl_pool: the span's first control point
    int64_t weight;  // floats into weight_pool: its first weight (NURBS), else -1
    int64_t dst;     // floats into span_pool: where the span is written
    int64_t op;      // entry of its extraction operator in op_pool (splines), else -1
    int32_t degree;
    int32_t type;    // bez_curve_type
    int64_t reserved;
};
static_assert(sizeof(SpanRec) == 48, "SpanRec is read as three 16-byte loads");

struct BatchArgs {
    const bez_curve_desc* desc;  // device copy
    int64_t n_curves;
    int32_t dim;
    const float* ctrl_pool;
    const float* weight_pool;
    float* out_pool;
    float* span_pool;            // every curve's spans in the evaluation representation
    const float2* op_pool;       // span operators M (repr 0) or T_p M (repr 1), each entry hi + lo (FP64 -> 2 x FP32),
                                 // row-major with rows padded to kOpRowStride(p) entries
    int64_t tpow_off[8];         // offset of T_p (Bezier -> centred power basis) in the centred op_pool
    const SpanRec* span_rec;     // every span, offsets resolved: one setup thread per component
    int64_t n_span_rec;
    int64_t span_class_start[16];  // spans of item class k: [span_class_start[k], span_class_start[k+1])
    int32_t repr;                // 0 Bezier points (de Casteljau), 1 power basis about 1/2 (Horner)
    const BatchItem* items;      // work items, sorted by item class
    int64_t n_items;
    int64_t class_start[16];     // items of class k: [class_start[k], class_start[k+1])
    int32_t chunk;
    int32_t schedule;            // 0 static round-robin, 1 atomic queue
    int32_t grab;                // items taken per atomic
    void* counter;               // one 8-byte work counter per class (atomic schedule)
    int32_t partition;           // atomic schedule: class k launches class_grid[k] blocks on a stream of its own
    int32_t class_grid[16];
};
// row stride (entries) of a degree-p extraction operator in the batch pool:
// p + 1 rounded up to even, so every row starts on a 16-byte boundary
__host__ __device__ constexpr int kOpRowStride(int p) { return (p + 1) + ((p + 1) & 1); }
// floats per span of degree p with `comps` components in the batch span pool:
// (p + 1) comps rounded up to a multiple of 4, so spans (whose pool offsets
// are multiples of 4 floats) load as whole float4s
__host__ __device__ constexpr int kSpanStride(int p, int comps) { return ((p + 1) * comps + 3) & ~3; }
constexpr int kBatchClasses = 15;  // 7 degrees x {integral, rational} for 3D curves + generic
int batch_item_class(const bez_curve_desc& d, int dim);
cudaError_t launch_batch(const BatchArgs& a, int threads, int sm_count, bool with_setup, cudaStream_t s,
                         const BatchStreams* bs, const LaunchHooks& h, int* launches);
// the grid a class kernel gets without partitioning (persistent: every SM full)
int batch_full_grid(const BatchArgs& a, int threads, int sm_count, int cls);

// Peak microbenchmarks (peaks.cu): kind 0 FP32 FMA lane-ops/s, 1..4 texture
// fetches/s (2D float4, 2D half4, 3D float4, 3D half4), 5 store GB/s,
// 6 copy GB/s.
cudaError_t measure_peak(int kind, int sm_count, cudaStream_t s, double* value);

// Message returned by bez_last_error() on the calling thread.
void set_last_error(const char* msg);

// Occupancy-sized persistent grid: a multiple of the SM count.
int persistent_grid(const void* kernel, int block, size_t smem, int sm_count, int64_t work_blocks);

}  // namespace bez
