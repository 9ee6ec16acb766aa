// noalloc.cu -- B-spline / NURBS evaluation that allocates no memory.
//
// bez_eval_bspline and bez_eval_nurbs keep the Bezier spans they extract in
// a scratch buffer that the context grows with cudaMalloc.  Some callers
// cannot allow that: code that must not synchronise the device (cudaMalloc
// and cudaFree can), hosts whose memory manager owns all device memory and
// forbids other allocations, and plugins that may only use the buffers they
// are handed.  bez_eval_spline_noalloc runs the same two kernels with the
// span scratch in a fixed array compiled into the library instead.
//
// The array is a file-scope __device__ symbol, so every GPU that loads the
// library holds kNoAllocSpanFloats floats (16 MiB) for the life of the
// process.  Host code cannot use the symbol's name as a device address; the
// address is looked up with cudaGetSymbolAddress once per device (on that
// device's first call, with the device current) and cached.  That first call
// should therefore come before any stream capture.  All calls share the
// array: calls that can overlap on the GPU (different streams without
// ordering) race on it.  Nothing in it has to start at zero: the setup
// kernel writes every span slot the evaluator reads, including empty spans.
// The call has no context, so its launches are not counted or timed by
// bez_get_stats.
#include <cstdio>
#include <mutex>

#include "../../include/bez.h"
#include "common.cuh"
#include "internal.h"

namespace {

constexpr size_t kNoAllocSpanFloats = size_t(4) << 20;  // 16 MiB of FP32 span control points
__device__ __align__(256) float g_span_scratch[kNoAllocSpanFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_scratch_ptr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};

void no_count(void*) {}
void no_event(void*, cudaStream_t) {}

bez_status fail_na(bez_status st, const char* msg)
{
    bez::set_last_error(msg);
    return st;
}

// device address of the scratch array on the current device (looked up once)
cudaError_t scratch_for_current_device(float** ptr, int* sm_count)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_ptr[dev]) {
        float* p = nullptr;
        e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_span_scratch);
        if (e != cudaSuccess) return e;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
        g_sm_count[dev] = sms;
    }
    *ptr = g_scratch_ptr[dev];
    *sm_count = g_sm_count[dev];
    return cudaSuccess;
}

// Whether p is device memory that kernels launched on device `dev` may
// read: memory allocated on `dev` itself, or managed memory.  A pointer to
// another GPU's memory is refused rather than dereferenced from the wrong
// device.
bool is_device_pointer_on(const void* p, int dev)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" bez_status bez_eval_spline_noalloc(const float* ctrl, const float* weights, const float* knots,
                                             int64_t n_curves, int n_ctrl, int degree, int dim, const float* t,
                                             int64_t n_t, float* out, const bez_opts* o, void* stream)
{
    using namespace bez;
    if (!o) return fail_na(BEZ_ERR_INVALID_ARG, "null opts");
    if (n_curves < 0 || n_t < 0) return fail_na(BEZ_ERR_INVALID_ARG, "negative size");
    if (n_t > 0x7fffffff) return fail_na(BEZ_ERR_INVALID_ARG, "n_t exceeds 2^31-1");
    if (dim < 1 || dim > 4) return fail_na(BEZ_ERR_INVALID_ARG, "dim not in 1..4");
    if (degree < 1 || n_ctrl < degree + 1) return fail_na(BEZ_ERR_INVALID_ARG, "need degree >= 1, n_ctrl >= degree+1");
    if (degree > kMaxDegree) return fail_na(BEZ_ERR_UNSUPPORTED, "degree above 15");
    if (o->dtype != BEZ_F32) return fail_na(BEZ_ERR_UNSUPPORTED, "splines take FP32 control points");
    if (o->out_mode < BEZ_OUT_POINTS || o->out_mode > BEZ_OUT_POLYLINE_LENGTH)
        return fail_na(BEZ_ERR_INVALID_ARG, "bad out_mode");
    if (o->t_mode < BEZ_T_SHARED || o->t_mode > BEZ_T_HASH) return fail_na(BEZ_ERR_INVALID_ARG, "bad t_mode");
    if (o->variant != BEZ_VAR_AUTO && o->variant != BEZ_VAR_DECASTELJAU)
        return fail_na(BEZ_ERR_UNSUPPORTED, "splines evaluate their Bezier spans by de Casteljau");
    if (o->t_mode == BEZ_T_HASH && n_curves > 0xffffffffLL)
        return fail_na(BEZ_ERR_INVALID_ARG, "hash parameters index curves with 32 bits");
    const int comps = weights ? dim + 1 : dim;
    const int64_t n_spans = n_ctrl - degree;
    const double need = (double)n_curves * (double)n_spans * (double)(degree + 1) * (double)comps;
    if (need > (double)kNoAllocSpanFloats) {
        char msg[200];
        snprintf(msg, sizeof(msg),
                 "batch needs %.0f span floats; the allocation-free entry point holds at most %zu (16 MiB)", need,
                 kNoAllocSpanFloats);
        return fail_na(BEZ_ERR_INVALID_ARG, msg);
    }
    if (n_curves == 0 || (n_t == 0 && o->out_mode == BEZ_OUT_POINTS)) return BEZ_OK;
    const bool t_array = o->t_mode == BEZ_T_SHARED || o->t_mode == BEZ_T_PER_CURVE;
    if (!ctrl || !out || (t_array && n_t > 0 && !t))
        return fail_na(BEZ_ERR_INVALID_ARG, "null ctrl, out or t");
    // this entry point stages nothing and switches no device: every array
    // must already be in the current device's memory
    int cur = 0;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return fail_na(BEZ_ERR_CUDA, cudaGetErrorString(e));
    if (!is_device_pointer_on(ctrl, cur) || !is_device_pointer_on(out, cur) ||
        (weights && !is_device_pointer_on(weights, cur)) || (knots && !is_device_pointer_on(knots, cur)) ||
        (t_array && n_t > 0 && !is_device_pointer_on(t, cur)))
        return fail_na(BEZ_ERR_INVALID_ARG,
                       "arrays must be device memory of the current device (host arrays would need staging "
                       "buffers; make the arrays' device current before the call)");

    float* scratch = nullptr;
    int sm_count = 0;
    e = scratch_for_current_device(&scratch, &sm_count);
    if (e != cudaSuccess) return fail_na(BEZ_ERR_CUDA, cudaGetErrorString(e));
    SplineArgs a{};
    a.ctrl = ctrl;
    a.weights = weights;
    a.knots = knots;
    a.n_curves = n_curves;
    a.n_ctrl = n_ctrl;
    a.degree = degree;
    a.dim = dim;
    a.comps = comps;
    a.n_spans = (int32_t)n_spans;
    a.spans = scratch;
    a.t = t_array ? t : nullptr;
    a.t_stride = o->t_mode == BEZ_T_PER_CURVE ? n_t : 0;
    a.n_t = (int32_t)n_t;
    a.out = out;
    a.err_word = o->err_word;
    const uint32_t seed_lo = (uint32_t)(o->seed & 0xffffffffu), seed_hi = (uint32_t)(o->seed >> 32);
    a.key = lowbias32(seed_lo ^ lowbias32(seed_hi ^ lowbias32(o->stream_id)));
    const int tm = t_array ? TM_ARRAY : (o->t_mode == BEZ_T_UNIFORM ? TM_UNIFORM : TM_HASH);
    const int om = o->out_mode == BEZ_OUT_POINTS ? OM_POINTS : OM_LENGTH;
    const LaunchHooks h{no_count, no_event, no_event, nullptr, sm_count};
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LaunchResult r = launch_spline_setup(a, s, h);
    if (r.err == cudaSuccess) r = launch_spline_eval(a, tm, om, s, h);
    if (r.err != cudaSuccess) return fail_na(BEZ_ERR_CUDA, cudaGetErrorString(r.err));
    if (o->sync) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail_na(BEZ_ERR_CUDA, cudaGetErrorString(e));
    }
    return BEZ_OK;
}
