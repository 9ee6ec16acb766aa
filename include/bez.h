/*
 * bez.h -- C ABI of libbez.so: batched evaluation of Bezier curves, C0
 * piecewise chains, B-splines / NURBS, tensor-product surfaces and volumes,
 * and the adjoint of curve evaluation, on an NVIDIA GB300 (sm_103a).
 *
 * The operations follow "A Texture Lookup Approach to Bezier Curve
 * Evaluation on the GPU" (Anas & Wolfe): a curve is evaluated at many
 * parameter values either in registers (power-basis Horner, Bernstein sum,
 * de Casteljau, Seiler interpolation) or by hardware-filtered texture lookups
 * of de Casteljau / Seiler control textures.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Arrays are contiguous, row-major, caller-owned.  A pointer may be device
 *   memory (cudaMalloc / torch CUDA tensor) or host memory (pageable or
 *   pinned).  Host arrays are staged through library-owned device buffers:
 *   inputs are copied in on `stream`, outputs copied back, and the call then
 *   synchronises `stream` before returning so the host output is valid.
 *   With device arrays only, calls are asynchronous on `stream` unless
 *   opts->sync is nonzero.  The library never frees or retains caller arrays.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 * - Argument errors are found on the host before any launch: the call returns
 *   BEZ_ERR_INVALID_ARG (or BEZ_ERR_UNSUPPORTED for a valid but unsupported
 *   variant / degree / dtype combination) and leaves outputs untouched.  A
 *   failed CUDA call returns BEZ_ERR_CUDA, a failed allocation BEZ_ERR_OOM;
 *   bez_last_error() gives the message.
 * - Parameters outside the domain are clamped to it (t in [0,1] for curves,
 *   [0,n_seg] for chains, [U_p, U_n] for splines); NaN propagates to the
 *   output.  Empty inputs (zero curves or zero samples) are valid no-ops.
 * - Outputs are FP32.  Control points are FP32 unless opts->dtype selects
 *   FP16 / BF16 storage (math stays FP32).
 */
#ifndef BEZ_H
#define BEZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum bez_status {
    BEZ_OK = 0,
    BEZ_ERR_INVALID_ARG = 1,
    BEZ_ERR_UNSUPPORTED = 2,
    BEZ_ERR_CUDA = 3,
    BEZ_ERR_OOM = 4,
    BEZ_ERR_TIMEOUT = 5
} bez_status;

/* Evaluator.  Register forms: paper Sec. 2 (de Casteljau as recursive lerps),
 * Sec. 3 (Seiler interpolation), Sec. 2.2 (power basis <-> Bernstein; the
 * "Polynomial" shader of Sec. 5).  Texture forms: Sec. 2 (de Casteljau
 * tiles), Sec. 4 (Seiler tiles), Fig. 3 (hybrid). */
typedef enum bez_variant {
    BEZ_VAR_AUTO = 0,            /* library choice: bez_eval takes HORNER_CENTRED up to  *
                                  * degree 7, SEILER above; chains, splines: DECASTELJAU */
    BEZ_VAR_HORNER = 1,          /* power basis about t=0, Horner, FP32 (baseline)       */
    BEZ_VAR_HORNER_CENTRED = 2,  /* power basis about t=1/2, Horner                      */
    BEZ_VAR_BERNSTEIN = 3,       /* Bernstein polynomial sum                             */
    BEZ_VAR_DECASTELJAU = 4,     /* de Casteljau, d(d+1)/2 lerps                          */
    BEZ_VAR_SEILER = 5,          /* Seiler interpolation, d lerps                         */
    BEZ_VAR_TEX_DECASTELJAU = 6, /* tex3D 2x2x2 de Casteljau tile (+ register levels)    */
    BEZ_VAR_TEX_SEILER = 7,      /* tex2D (d=2,3) / tex3D (d=4..7) Seiler tile           */
    BEZ_VAR_TEX_HYBRID = 8,      /* two bilinear reads + FP32 lerp (cubic)               */
    BEZ_VAR_TENSOR = 9,          /* reserved (tensor-core grid contraction, not built:   *
                                  * the grid kernels are bound by their stores)          */
    BEZ_VAR_COISSUE = 10,        /* tex2D Seiler for opts->tex_share of every 8 samples, *
                                  * centred Horner for the rest, in one kernel           */
    BEZ_VAR_HALF2 = 11           /* centred Horner in half2 arithmetic (FP16 math, two   *
                                  * samples per instruction), dim 3, degree 1..7         */
} bez_variant;

typedef enum bez_dtype { BEZ_F32 = 0, BEZ_F16 = 1, BEZ_BF16 = 2 } bez_dtype;

typedef enum bez_out_mode {
    BEZ_OUT_POINTS = 0,          /* out [n_curves][n_t][dim]                              */
    BEZ_OUT_POLYLINE_LENGTH = 1  /* out [n_curves] = sum_{j>=1} |P_j - P_{j-1}|, FP32 acc */
} bez_out_mode;

typedef enum bez_t_mode {
    BEZ_T_SHARED = 0,    /* t [n_t], same parameters for every curve                   */
    BEZ_T_PER_CURVE = 1, /* t [n_curves][n_t]                                          */
    BEZ_T_UNIFORM = 2,   /* t_j = fl32(j) / fl32(n_t - 1) (0 when n_t == 1); t unused   */
    BEZ_T_HASH = 3       /* t drawn in-kernel (lowbias32 counter hash of seed, stream,   *
                          * curve, j); t unused.  See bez_eval.                         */
} bez_t_mode;

/* Texel format of texture tiles.  AUTO: float4 for FP32 control points,
 * half4 for FP16.  UNORM16 / UNORM8 (Sec. 2.3: low-bit-depth texels hold
 * [0, 1]): each curve's tile is stored as (texel - lo) / scale per component,
 * lo and scale its tile's minimum and range, and the filtered value is mapped
 * back by lo + scale * f; texel rounding adds 2^-17 (16-bit) or 2^-9 (8-bit)
 * of the tile's range to the 8-bit filter-weight error. */
typedef enum bez_tex_format {
    BEZ_TEX_AUTO = 0,
    BEZ_TEX_UNORM16 = 1,
    BEZ_TEX_UNORM8 = 2
} bez_tex_format;

typedef struct bez_opts {
    int32_t variant;   /* bez_variant                                                   */
    int32_t dtype;     /* bez_dtype of the control points                               */
    int32_t out_mode;  /* bez_out_mode                                                  */
    int32_t t_mode;    /* bez_t_mode                                                    */
    uint64_t seed;     /* BEZ_T_HASH only                                               */
    uint32_t stream_id;/* BEZ_T_HASH only: independent parameter stream under one seed  */
    int32_t sync;      /* nonzero: synchronise `stream` before returning                 */
    int32_t* err_word; /* device int32 or NULL: incremented for data faults (NURBS zero  *
                        * denominators)                                                 */
    int32_t tex_share; /* BEZ_VAR_COISSUE only: samples out of every 8 read through the  *
                        * texture unit, 1..7; 0 = library default (2)                    */
    int32_t tex_format;/* bez_tex_format of texture tiles of bez_eval (texture variants   *
                        * and BEZ_VAR_COISSUE) and of bez_eval_surface (texture           *
                        * variants); texture chains take BEZ_TEX_AUTO only; entry points  *
                        * and variants without textures ignore it                         */
    int32_t tex_spread;/* 0 or 1: the paper's tile layouts.  2, 4, 8, 16 (s): spread     *
                        * tiles, each 2D tile's bilinear function sampled on (s+1) x      *
                        * (s+1) texels and read at s times its coordinates, which cuts   *
                        * the error of the 8-bit filter weights about s-fold (Sec. 2.3)  *
                        * for (s+1)^2 / 4 times the texture memory.  Built for           *
                        * BEZ_VAR_TEX_SEILER curves of degree 2, 3 (bez_eval), the       *
                        * zig-zag chain texture (bez_eval_piecewise) and TEX_SEILER      *
                        * surfaces and volumes; elsewhere a value above 1 returns        *
                        * BEZ_ERR_UNSUPPORTED.  Other values: BEZ_ERR_INVALID_ARG.       */
} bez_opts;

/* Opaque context: owns staging buffers, texture atlases, timing events. */
typedef struct bez_ctx_s* bez_ctx;

/* Create a context on CUDA device `device` (makes it current on this thread). */
bez_status bez_create(bez_ctx* ctx, int device);
/* Destroy a context and everything it owns; waits for its pending work. */
bez_status bez_destroy(bez_ctx ctx);
/* Message for the last non-OK status returned on the calling thread. */
const char* bez_last_error(void);
/* Library version string. */
const char* bez_version(void);

/* Launch accounting.  `launches` counts every kernel this context launched
 * since the last reset.  With timing enabled, the main evaluator kernel of
 * every call is bracketed by CUDA events on the launching stream;
 * bez_get_stats waits for those events and reports their count and summed
 * duration. */
typedef struct bez_stats {
    int64_t launches;
    int64_t timed_launches;
    double timed_ms;
} bez_stats;
bez_status bez_set_timing(bez_ctx ctx, int enable);
bez_status bez_get_stats(bez_ctx ctx, bez_stats* out);
bez_status bez_reset_stats(bez_ctx ctx);

/*
 * bez_eval -- Bezier curves at many parameters.
 *
 * Paper Sec. 2 (de Casteljau recursion, pixel-centre t remap), Sec. 2.2
 * (power basis <-> Bernstein), Sec. 3 (Seiler interpolation, arbitrary
 * degree via the difference terms d_i), Sec. 4 (Seiler textures).
 *
 *   ctrl  [n_curves][degree+1][dim], element type opts->dtype
 *   t     per opts->t_mode (NULL for UNIFORM / HASH)
 *   out   POINTS: [n_curves][n_t][dim] FP32;  POLYLINE_LENGTH: [n_curves] FP32
 *   degree 1..15 (texture Seiler: 2..7); dim 1..4.
 *
 * Texture variants pack the control points into a cudaArray atlas owned by
 * the context (one surface-write kernel), then evaluate with hardware linear
 * filtering (one kernel).  Seiler tiles: the paper's layouts for degrees 2..5
 * (read at (t, st) and (t, st, st)); for degrees 6, 7 a 2x2x2 tile holding
 * L(d_k, d_(d-k), t) / 4^k in its corners, read at (t, 4 st, 16 st^2).  dtype F32 gives float4 texels, F16 half4 texels;
 * BF16 has no texture format (BEZ_ERR_UNSUPPORTED).  Calls of one context
 * that use the atlases are ordered across streams by the library.
 *
 * BEZ_T_HASH draws t_(c,j) = (h >> 9) * 2^-23 with
 *   h = H(H(key ^ c) ^ j),  key = H(lo(seed) ^ H(hi(seed) ^ H(stream_id))),
 *   H = lowbias32 (Wellons 2018: x^=x>>16; x*=0x7feb352d; x^=x>>15;
 *   x*=0x846ca68b; x^=x>>16), c < 2^32, j < 2^32.
 *
 * BEZ_VAR_HALF2: the centred power basis (FP32 setup, FP64 from degree 5)
 * rounded to half; a lane evaluates two samples per HFMA2.  Parameters are
 * drawn and lengths accumulated in FP32.  Accuracy is that of 11-bit
 * arithmetic (about 1e-3 of the curve size for cubics), far from the FP32
 * forms; dim 3 and degrees 1..7 only (else BEZ_ERR_UNSUPPORTED).
 *
 * BEZ_VAR_COISSUE (Sec. 5: a texture read pays off when it overlaps
 * arithmetic): cubic 3D curves, POLYLINE_LENGTH, BEZ_T_HASH with
 * n_t <= 65536, dtype F32 or F16.  In every group of 8 consecutive samples
 * of a lane's run, the first opts->tex_share samples are read from the
 * curve's tex2D Seiler tile and the rest are evaluated by centred Horner in
 * registers, so the texture unit and the FP32 pipes work side by side.
 * Accuracy is that of the texture reads.  Other combinations return
 * BEZ_ERR_UNSUPPORTED.
 */
bez_status bez_eval(bez_ctx ctx, const void* ctrl, int64_t n_curves, int degree, int dim,
                    const float* t, int64_t n_t, float* out, const bez_opts* opts, void* stream);

/*
 * bez_eval_piecewise -- C0 piecewise Bezier chains.
 *
 * Paper Sec. 2.1 (Eq. 1-2, Fig. 2): consecutive segments share end points;
 * a quadratic chain of N segments fits an (N+1) x 2 texture because the two
 * diagonal texels of each 2x2 window only need to average to the middle
 * control point, and the texture is read along a zig-zag path.
 *
 *   ctrl  [n_chains][n_seg*degree+1][dim] logical control points (segment k
 *         uses points k*degree .. k*degree+degree), element type opts->dtype
 *   t     global parameters in [0, n_seg] per opts->t_mode; segment
 *         k = min(floor(t), n_seg-1), local parameter t - k.  UNIFORM gives
 *         t_j = fl32(n_seg * fl32(j)/fl32(n_t-1)); HASH gives
 *         t = fl32(n_seg * u) with u the bez_eval draw.
 *   out   POINTS [n_chains][n_t][dim] or POLYLINE_LENGTH [n_chains], FP32
 *
 * BEZ_VAR_TEX_DECASTELJAU evaluates quadratic chains (degree 2) from the
 * zig-zag texture; the free texel of each chain is chosen per component to
 * minimise the largest texel magnitude.  The read snaps the fraction both
 * axes share to the filter's 1/256 grid, so both weights round alike;
 * opts->tex_spread s >= 2 samples each 2x2 window on (s+1) x (s+1) texels
 * (an (N s + 1) x (s + 1) texture) for about s times less weight error.
 * Texels are float4 (FP32 control points), half4 (F16), or, with
 * opts->tex_format BEZ_TEX_UNORM16 and FP32 control points, unorm16 codes
 * of each chain's per-component texel range (Sec. 2.3's low-bit-depth
 * formats; the filtered value is mapped back by the range, adding at most
 * range / 131070 per component); BEZ_TEX_UNORM8 returns
 * BEZ_ERR_UNSUPPORTED (the free texels span tens of the control points'
 * extent).  Cubic chains (degree 3; Sec. 2.1: two quadratic chains front to back in a
 * 3D texture) use an (N+1) x 2 x 2 texture read trilinearly along a 3D
 * zig-zag: the three texels one flip from a segment's corner average to its
 * second control point and the three two flips away to its third; spread 0
 * or 1 only.  Register variants take any degree
 * 1..15 with (n_seg*degree+1)*dim <= 3072; the chain is staged in shared
 * memory.  Default (AUTO): register de Casteljau.
 */
bez_status bez_eval_piecewise(bez_ctx ctx, const void* ctrl, int64_t n_chains, int n_seg, int degree, int dim,
                              const float* t, int64_t n_t, float* out, const bez_opts* opts, void* stream);

/*
 * bez_eval_bspline / bez_eval_nurbs -- B-spline and NURBS curves.
 *
 * Paper Sec. 2.2: B-splines become piecewise Bezier curves by Boehm's knot
 * insertion, and rational curves divide one integral spline point by
 * another (homogeneous coordinates).  A setup kernel extracts the Bezier
 * control points of every span in FP64 (one thread per span; rational
 * curves in homogeneous form (w P, w)) into a library-owned scratch buffer;
 * the evaluator finds each parameter's span, runs FP32 de Casteljau on it
 * and, for NURBS, divides by the weight.
 *
 *   ctrl     [n_curves][n_ctrl][dim] FP32 (opts->dtype must be BEZ_F32)
 *   weights  [n_curves][n_ctrl] FP32 (NURBS only; positive weights expected)
 *   knots    [n_curves][n_ctrl+degree+1] FP32, nondecreasing, or NULL for the
 *            clamped uniform vector (degree+1 zeros, i/(n_ctrl-degree),
 *            degree+1 ones)
 *   t        knot-space parameters per opts->t_mode, clamped to
 *            [U_degree, U_n_ctrl]; UNIFORM / HASH map their [0,1] draws
 *            affinely onto that domain.  A parameter on an interior knot
 *            belongs to the later span.
 *   out      POINTS [n_curves][n_t][dim] or POLYLINE_LENGTH [n_curves], FP32
 *   degree 1..15, n_ctrl >= degree+1, dim 1..4; variant AUTO or
 *   DECASTELJAU.  A zero rational denominator increments *opts->err_word.
 */
bez_status bez_eval_bspline(bez_ctx ctx, const float* ctrl, const float* knots, int64_t n_curves, int n_ctrl,
                            int degree, int dim, const float* t, int64_t n_t, float* out, const bez_opts* opts,
                            void* stream);
bez_status bez_eval_nurbs(bez_ctx ctx, const float* ctrl, const float* weights, const float* knots, int64_t n_curves,
                          int n_ctrl, int degree, int dim, const float* t, int64_t n_t, float* out,
                          const bez_opts* opts, void* stream);

/*
 * bez_eval_surface / bez_eval_volume -- tensor-product Bezier surfaces and
 * volumes on uniform parameter grids.
 *
 * Paper Sec. 2.2: a surface splits its order between u and v (a bicubic
 * patch evaluates its four column curves at u, giving the control points of
 * the isoline cubic in v); a volume splits it between u, v and w.  The
 * kernels contract separably (columns at u, then v, then w) with Bernstein
 * tables of the grid values fl32(a)/fl32(n-1) (one warp per patch for
 * bicubic 3D patches with nu <= 64, else one block per patch), and write
 * the output with coalesced (float4 where aligned) stores.
 *
 *   surface ctrl [n][du+1][dv+1][dim]        -> out [n][nu][nv][dim]
 *   volume  ctrl [n][du+1][dv+1][dw+1][dim]  -> out [n][nu][nv][nw][dim]
 *   degrees 1..7, grid sizes 1..256 per axis, dim 1..4; ctrl element type
 *   opts->dtype (FP32, FP16 or BF16 storage, FP32 math); out_mode POINTS;
 *   t_mode and t are not used.
 *   variant AUTO or BERNSTEIN: FP32 contraction on CUDA cores.
 *   variant TEX_DECASTELJAU (bicubic surfaces, nu <= 64, FP32 or FP16
 *   storage): per patch and coordinate a 2x2x2 RGBA texture tile holds the
 *   four column cubics (Sec. 2.2); one trilinear read at (u,u,u) per grid
 *   row gives the isoline control points, the cubic in v runs in FP32.
 *   variant TEX_SEILER (same limits): the four column cubics in the 2x2
 *   cubic Seiler layout (Sec. 4), one per channel of a 2D tile, read
 *   bilinearly at (u, u (1 - u)); with opts->tex_spread s >= 2 each
 *   channel's Seiler function is sampled on an (s+1) x (s+1) tile read at
 *   (s u, 4 s u (1 - u)), which divides the filter-weight error by about s.
 *   bez_eval_volume with TEX_DECASTELJAU / TEX_SEILER: tricubic scalar
 *   volumes (dim 1, nu <= 32, nw a multiple of 4, out 16-byte aligned);
 *   tile (p, j) holds the u cubics C[.][j][l] in channel l, one read per
 *   (row u, j), v and w contract in FP32.
 *   Texels are float4 (FP32 input) or half4 (FP16 input), or with
 *   opts->tex_format UNORM16 / UNORM8 16- or 8-bit codes with one (lo,
 *   scale) pair per tile and channel, mapped back after filtering as for
 *   curves.  Accuracy is that of 8-bit filter weights (about 3 x 2^-8 of the
 *   column range) plus half a code of the tile's range for unorm texels; the
 *   tiles live in a context-owned atlas, so texture calls of one context are
 *   ordered on the device.  Other combinations return BEZ_ERR_UNSUPPORTED.
 */
bez_status bez_eval_surface(bez_ctx ctx, const void* ctrl, int64_t n, int du, int dv, int dim, int nu, int nv,
                            float* out, const bez_opts* opts, void* stream);
bez_status bez_eval_volume(bez_ctx ctx, const void* ctrl, int64_t n, int du, int dv, int dw, int dim, int nu, int nv,
                           int nw, float* out, const bez_opts* opts, void* stream);

/*
 * Mixed batches -- curves of different type, degree and sample count in one
 * persistent launch (the batching pattern the paper's evaluators need when a
 * scene mixes curve kinds; the curve types are those of Sec. 2.2).
 *
 * Each curve has a descriptor.  Control points of curve c are
 * ctrl_pool[ctrl_off .. ctrl_off + n_ctrl*dim); NURBS weights
 * weight_pool[weight_off .. + n_ctrl); its points go to
 * out_pool[out_off .. out_off + n_samples*dim), evaluated at
 * t_j = fl32(j) / fl32(n_samples - 1) over the curve's domain [0, 1].
 *   BEZ_CURVE_BEZIER  n_ctrl == degree + 1
 *   BEZ_CURVE_BSPLINE clamped uniform knots, n_ctrl >= degree + 1
 *   BEZ_CURVE_NURBS   clamped uniform knots and weights
 *   degree 1..7, dim 1..4; pools are FP32 device arrays of the stated
 *   lengths (in floats); descriptors are host or device arrays.
 *
 * bez_batch_create validates every descriptor on the host (offsets against
 * the pool lengths), builds the work-item table (curve, chunk of samples),
 * computes the FP64 knot-insertion operators of every distinct (n_ctrl,
 * degree) of the splines, allocates the plan's device buffers (descriptors,
 * items, operators, the span pool), optionally autotunes the span
 * representation (Bezier points / power basis about 1/2), chunk size,
 * scheduler (static round-robin or atomic work queue) and block size by
 * timing candidates on the real batch (results cached in memory and, when
 * the environment variable BEZ_AUTOTUNE_CACHE names a file, in that JSON
 * file), and captures span setup + evaluation in a CUDA graph.
 * bez_batch_launch replays it on `stream`; with setup_each_launch = 0 the
 * spans are extracted once at creation (control points must then not
 * change).  bez_eval_batch is create + launch + destroy without graph or
 * tuning, synchronous on `stream`.
 */
typedef enum bez_curve_type { BEZ_CURVE_BEZIER = 0, BEZ_CURVE_BSPLINE = 1, BEZ_CURVE_NURBS = 2 } bez_curve_type;

typedef struct bez_curve_desc {
    int32_t type;       /* bez_curve_type */
    int32_t degree;
    int32_t n_ctrl;
    int32_t n_samples;
    int64_t ctrl_off;   /* floats into ctrl_pool   */
    int64_t weight_off; /* floats into weight_pool */
    int64_t out_off;    /* floats into out_pool    */
} bez_curve_desc;

typedef struct bez_batch_opts {
    int32_t autotune;          /* time candidate launch shapes at creation      */
    int32_t setup_each_launch; /* re-extract spline spans on every launch        */
    int32_t use_graph;         /* capture setup + evaluation in a CUDA graph     */
    int32_t chunk;             /* samples per work item (multiple of 256), 0 = default / tuned */
    int32_t schedule;          /* -1 default / tuned, 0 static, 1 atomic queue,   *
                                * 2 atomic queue with the GPU partitioned between *
                                * the curve classes: every class kernel on its own *
                                * stream with a grid sized to its share of the     *
                                * work, measured per class at creation, so all     *
                                * classes run side by side and finish together    */
    int32_t threads;           /* threads per block (128, 256), 0 = default / tuned */
    int32_t repr;              /* -1 default / tuned, 0 Bezier points (de Casteljau),
                                * 1 power basis about 1/2 (Horner)              */
} bez_batch_opts;

typedef struct bez_batch_s* bez_batch;

bez_status bez_batch_create(bez_ctx ctx, const bez_curve_desc* desc, int64_t n_curves, int dim,
                            const float* ctrl_pool, int64_t ctrl_len, const float* weight_pool, int64_t weight_len,
                            float* out_pool, int64_t out_len, const bez_batch_opts* bopts, void* stream,
                            bez_batch* batch);
bez_status bez_batch_launch(bez_batch batch, void* stream);
/* chosen launch shape: chunk, schedule (0 static, 1 atomic, 2 atomic partitioned), threads,
 * span representation */
bez_status bez_batch_config(bez_batch batch, int32_t* chunk, int32_t* schedule, int32_t* threads, int32_t* repr);
bez_status bez_batch_destroy(bez_batch batch);
bez_status bez_eval_batch(bez_ctx ctx, const bez_curve_desc* desc, int64_t n_curves, int dim, const float* ctrl_pool,
                          int64_t ctrl_len, const float* weight_pool, int64_t weight_len, float* out_pool,
                          int64_t out_len, void* stream);

/*
 * bez_eval_backward -- adjoint of (rational) Bezier curve evaluation.
 *
 * Differentiates C(t) = sum_i B_i(t) w_i P_i / sum_i B_i(t) w_i (w = 1 when
 * weights is NULL; the rational form is Sec. 2.2's quotient of two integral
 * curves) for an upstream gradient grad_out = dL/dC(t_j):
 *   grad_ctrl[c][i]    = sum_j (w_i B_i(t_j) / W_j) grad_out[c][j]
 *   grad_weights[c][i] = sum_j B_i(t_j) (P_i - C(t_j)) . grad_out[c][j] / W_j
 *   grad_t[c][j]       = grad_out[c][j] . C'(t_j), 0 where t_j was clamped
 *                        (shared t: summed over curves, grad_t [n_t])
 *
 *   ctrl [n_curves][degree+1][dim] FP32, weights [n_curves][degree+1] or NULL
 *   t    SHARED [n_t] or PER_CURVE [n_curves][n_t] (opts->t_mode)
 *   grad_out [n_curves][n_t][dim]
 *   Outputs are overwritten; any of grad_ctrl, grad_weights, grad_t may be
 *   NULL (grad_weights needs weights).  degree 1..15, dim 1..4.
 */
bez_status bez_eval_backward(bez_ctx ctx, const float* ctrl, const float* weights, int64_t n_curves, int degree,
                             int dim, const float* t, int64_t n_t, const float* grad_out, float* grad_ctrl,
                             float* grad_weights, float* grad_t, const bez_opts* opts, void* stream);

/*
 * bez_mse_grad -- squared-error fit loss and its gradients in one pass.
 *
 * The paper has no counterpart; this is the curve-fitting step of the
 * differentiation workload with the loss fused into bez_eval_backward: for
 * targets y[c][j] and s = loss_scale,
 *   loss[c]       = s * sum_j ||C(t_j) - y_j||^2
 *   grad_*        = bez_eval_backward's outputs for grad_out = 2 s (C - y)
 * computed from the curve values the adjoint forms anyway, so the call reads
 * t and the targets once and writes no point or gradient arrays.
 *
 *   target [n_curves][n_t][dim] FP32; loss [n_curves] FP32 or NULL; other
 *   arguments, layouts and limits as bez_eval_backward.  Pass s =
 *   1 / (n_curves n_t dim) for the mean squared error.
 */
bez_status bez_mse_grad(bez_ctx ctx, const float* ctrl, const float* weights, int64_t n_curves, int degree, int dim,
                        const float* t, int64_t n_t, const float* target, float loss_scale, float* loss,
                        float* grad_ctrl, float* grad_weights, float* grad_t, const bez_opts* opts, void* stream);

/*
 * bez_eval_spline_noalloc -- B-spline / NURBS evaluation that allocates no
 * memory.  The paper has no counterpart; this is a deployment variant of
 * bez_eval_bspline / bez_eval_nurbs.
 *
 * Those calls keep the Bezier spans they extract in a scratch buffer that
 * the context grows with cudaMalloc.  Some callers cannot allow that: code
 * that must never synchronise the device (cudaMalloc / cudaFree can), hosts
 * whose memory manager owns all device memory, and plugins that may only use
 * the buffers they are given.  This entry point runs the same kernels with
 * the span scratch in a fixed 16 MiB array built into the library, which
 * every GPU that loads the library holds until the process exits.
 *
 *   weights NULL evaluates B-splines, non-NULL NURBS; other arguments as in
 *   bez_eval_nurbs, with no context.  Every array must be device memory of
 *   the calling thread's current device (or managed memory): host arrays
 *   would need staging buffers, and the call never switches devices, so
 *   arrays of another GPU are refused.  BEZ_ERR_INVALID_ARG otherwise.
 *   The batch may need at most 4,194,304 span floats,
 *   n_curves * (n_ctrl - degree) * (degree + 1) * (dim, or dim+1 for NURBS);
 *   larger batches are rejected with BEZ_ERR_INVALID_ARG.
 *
 * The first call on a device looks up the array's device address with that
 * device current; make it before any stream capture.  All calls share the
 * array and each overwrites it, so calls that may overlap on the GPU
 * (different streams without ordering between them) race.  Errors are
 * reported through bez_last_error().  Having no context, the call's
 * launches are not counted or timed by bez_get_stats.
 */
bez_status bez_eval_spline_noalloc(const float* ctrl, const float* weights, const float* knots, int64_t n_curves,
                                   int n_ctrl, int degree, int dim, const float* t, int64_t n_t, float* out,
                                   const bez_opts* opts, void* stream);

/*
 * bez_measure_peak -- microbenchmarks giving the roofline denominators of the
 * evaluators on this device (no counterpart in the paper, whose Sec. 5 times
 * whole frames).  Synchronous; allocates and frees its own buffers.
 *   BEZ_PEAK_FMA      FP32 FMA lane operations per second (8 independent
 *                     chains per thread, every SM busy)
 *   BEZ_PEAK_TEX2D_F32 / _F16  bilinear-filtered float4 / half4 fetches per
 *                     second from an L1-resident 64x64 texture
 *   BEZ_PEAK_TEX3D_F32 / _F16  trilinear-filtered fetches per second
 *   BEZ_PEAK_STORE    device-memory store bandwidth, GB/s (2 GiB of float4)
 *   BEZ_PEAK_COPY     device-memory copy bandwidth, GB/s counting read+write
 */
typedef enum bez_peak_kind {
    BEZ_PEAK_FMA = 0,
    BEZ_PEAK_TEX2D_F32 = 1,
    BEZ_PEAK_TEX2D_F16 = 2,
    BEZ_PEAK_TEX3D_F32 = 3,
    BEZ_PEAK_TEX3D_F16 = 4,
    BEZ_PEAK_STORE = 5,
    BEZ_PEAK_COPY = 6
} bez_peak_kind;
bez_status bez_measure_peak(bez_ctx ctx, int kind, double* value, void* stream);

/*
 * bez_probe_filter -- characterise the texture unit's linear-filter weights.
 *
 * Paper Sec. 2.3: the hardware converts texture coordinates to a fixed-point
 * format with 8 fractional bits before interpolating, which bounds the
 * accuracy of every texture evaluator.  This call samples a 2x2x2 float4
 * texture whose texel (x,y,z) holds (x, y, z, 1) with linear filtering and
 * clamp addressing: at unnormalised coordinates (X, Y, Z) the first three
 * channels return the total weight given to the texels with index 1 along
 * each axis, and the fourth the sum of all eight texel weights.
 *
 *   xyz  [n][3] FP32 coordinates (texel centres at 0.5 and 1.5)
 *   out  [n][4] FP32 filtered values
 */
bez_status bez_probe_filter(bez_ctx ctx, const float* xyz, int64_t n, float* out, void* stream);

/*
 * bez_probe_filter_2d -- the four texel weights of one bilinear read.
 *
 * Paper Sec. 2.3 (8-bit fractional filter weights).  Samples a 2x2 float4
 * texture whose texel (x, y) holds the unit vector of channel x + 2 y, with
 * linear filtering and clamp addressing, so the read at unnormalised
 * coordinates (X, Y) returns the weights w00, w10, w01, w11 the hardware
 * gives the four texels.  On GB300 they follow one rule: a = round8(frac(X -
 * 0.5)), b = round8(frac(Y - 0.5)) (round to nearest 1/256, ties up), w11 =
 * round8(a b), w10 = a - w11, w01 = b - w11, w00 = 1 - a - b + w11.
 *
 *   xy   [n][2] FP32 coordinates (texel centres at 0.5 and 1.5)
 *   out  [n][4] FP32 weights (w00, w10, w01, w11); synchronous
 */
bez_status bez_probe_filter_2d(bez_ctx ctx, const float* xy, int64_t n, float* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BEZ_H */
