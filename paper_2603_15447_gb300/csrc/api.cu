// api.cu -- host runtime of libbez.so: contexts, argument validation, host
// staging, launch accounting and dispatch to the kernels.  The C ABI is
// declared in include/bez.h.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <map>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/bez.h"
#include "context.h"
#include "internal.h"

using namespace bez;

#include "common.cuh"

// ---------------------------------------------------------------- errors

static thread_local std::string g_last_error;

bez_status bez::fail(bez_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

bez_status bez::cuda_fail(cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation) return fail(BEZ_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(BEZ_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

namespace bez {
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace bez

// ---------------------------------------------------------------- context

namespace {

cudaEvent_t take_event(bez_ctx c)
{
    if (!c->spare.empty()) {
        cudaEvent_t e = c->spare.back();
        c->spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void hook_count(void* self) { static_cast<bez_ctx>(self)->launches += 1; }

void hook_begin(void* self, cudaStream_t s)
{
    bez_ctx c = static_cast<bez_ctx>(self);
    if (!c->timing) return;
    c->cur_begin = take_event(c);
    cudaEventRecord(c->cur_begin, s);
}

void hook_end(void* self, cudaStream_t s)
{
    bez_ctx c = static_cast<bez_ctx>(self);
    if (!c->timing || !c->cur_begin) return;
    cudaEvent_t e = take_event(c);
    cudaEventRecord(e, s);
    c->pending.emplace_back(c->cur_begin, e);
    c->cur_begin = nullptr;
}

}  // namespace

LaunchHooks bez::hooks_of(bez_ctx c) { return LaunchHooks{hook_count, hook_begin, hook_end, c, c->sm_count}; }

bez::MemKind bez::classify(const void* p)
{
    if (!p) return MEM_NULL;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MEM_HOST;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? MEM_DEVICE : MEM_HOST;
}

namespace {

bez_status ensure_stage(bez_ctx c, int slot, size_t bytes, cudaStream_t s)
{
    StageBuf& b = c->stage[slot];
    if (b.cap >= bytes) return BEZ_OK;
    if (b.p) {
        BEZ_CUDA(cudaStreamSynchronize(s), "staging resize sync");
        BEZ_CUDA(cudaFree(b.p), "cudaFree staging");
        b.p = nullptr;
        b.cap = 0;
    }
    size_t cap = bytes < (1u << 20) ? (1u << 20) : bytes + bytes / 4;
    BEZ_CUDA(cudaMalloc(&b.p, cap), "cudaMalloc staging");
    b.cap = cap;
    return BEZ_OK;
}

// Staging plan of one call: host arrays are copied to device buffers owned by
// the context, outputs are copied back after the kernels.
struct Staging {
    bez_ctx c;
    cudaStream_t s;
    bool any_host = false;
    struct Out {
        void* host;
        void* dev;
        size_t bytes;
    };
    std::vector<Out> outs;

    Staging(bez_ctx ctx, cudaStream_t stream) : c(ctx), s(stream) {}

    bez_status in(const void* p, size_t bytes, int slot, const void** dev)
    {
        MemKind k = classify(p);
        if (k != MEM_HOST) {
            *dev = p;
            return BEZ_OK;
        }
        any_host = true;
        if (bytes == 0) {
            *dev = p;
            return BEZ_OK;
        }
        bez_status st = ensure_stage(c, slot, bytes, s);
        if (st != BEZ_OK) return st;
        BEZ_CUDA(cudaMemcpyAsync(c->stage[slot].p, p, bytes, cudaMemcpyHostToDevice, s), "copy input to device");
        *dev = c->stage[slot].p;
        return BEZ_OK;
    }

    bez_status out(void* p, size_t bytes, int slot, void** dev)
    {
        MemKind k = classify(p);
        if (k != MEM_HOST) {
            *dev = p;
            return BEZ_OK;
        }
        any_host = true;
        if (bytes == 0) {
            *dev = p;
            return BEZ_OK;
        }
        bez_status st = ensure_stage(c, slot, bytes, s);
        if (st != BEZ_OK) return st;
        *dev = c->stage[slot].p;
        outs.push_back({p, c->stage[slot].p, bytes});
        return BEZ_OK;
    }

    bez_status finish(int sync)
    {
        for (auto& o : outs)
            BEZ_CUDA(cudaMemcpyAsync(o.host, o.dev, o.bytes, cudaMemcpyDeviceToHost, s), "copy output to host");
        if (any_host || sync) BEZ_CUDA(cudaStreamSynchronize(s), "stream synchronize");
        return BEZ_OK;
    }
};

size_t dtype_size(int dt) { return dt == BEZ_F32 ? 4 : 2; }

// pipelined host calls: at most kPipeChunks chunks of at least kPipeMinCurves curves
constexpr int kPipeChunks = 8;
static_assert(sizeof(((bez_ctx_s*)nullptr)->pipe_ev) / sizeof(cudaEvent_t) == 2 * kPipeChunks + 2,
              "one start event, an in and a done event per chunk, one end event");
constexpr int64_t kPipeMinCurves = 16384;

bez_status check_common(bez_ctx c, const bez_opts* o)
{
    if (!c) return fail(BEZ_ERR_INVALID_ARG, "null context");
    if (!o) return fail(BEZ_ERR_INVALID_ARG, "null opts");
    if (o->dtype < BEZ_F32 || o->dtype > BEZ_BF16) return fail(BEZ_ERR_INVALID_ARG, "bad dtype %d", o->dtype);
    if (o->out_mode < BEZ_OUT_POINTS || o->out_mode > BEZ_OUT_POLYLINE_LENGTH)
        return fail(BEZ_ERR_INVALID_ARG, "bad out_mode %d", o->out_mode);
    if (o->t_mode < BEZ_T_SHARED || o->t_mode > BEZ_T_HASH) return fail(BEZ_ERR_INVALID_ARG, "bad t_mode %d", o->t_mode);
    if (o->variant < BEZ_VAR_AUTO || o->variant > BEZ_VAR_HALF2)
        return fail(BEZ_ERR_INVALID_ARG, "bad variant %d", o->variant);
    if (o->tex_format < BEZ_TEX_AUTO || o->tex_format > BEZ_TEX_UNORM8)
        return fail(BEZ_ERR_INVALID_ARG, "bad tex_format %d", o->tex_format);
    if (o->tex_spread < 0 || o->tex_spread > 16 || (o->tex_spread & (o->tex_spread - 1)) != 0)
        return fail(BEZ_ERR_INVALID_ARG, "tex_spread %d is not 0 or a power of two up to 16", o->tex_spread);
    return BEZ_OK;
}

}  // namespace

namespace bez {

int persistent_grid(const void* kernel, int block, size_t smem, int sm_count, int64_t work_blocks)
{
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, size_t>, int> cache;
    const auto key = std::make_tuple(kernel, block, smem);
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find(key);
        if (it != cache.end()) per_sm = it->second;
    }
    if (per_sm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        std::lock_guard<std::mutex> g(mu);
        cache[key] = per_sm;
    }
    int64_t full = (int64_t)per_sm * sm_count;
    if (work_blocks < 1) work_blocks = 1;
    return (int)(work_blocks < full ? work_blocks : full);
}

}  // namespace bez

// ---------------------------------------------------------------- C ABI

extern "C" {

const char* bez_version(void) { return "bez 0.1 (sm_103a)"; }

const char* bez_last_error(void) { return g_last_error.c_str(); }

bez_status bez_create(bez_ctx* out, int device)
{
    if (!out) return fail(BEZ_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    int n = 0;
    BEZ_CUDA(cudaGetDeviceCount(&n), "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(BEZ_ERR_INVALID_ARG, "device %d out of range (%d devices)", device, n);
    BEZ_CUDA(cudaSetDevice(device), "cudaSetDevice");
    cudaDeviceProp prop;
    BEZ_CUDA(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");
    if (prop.major < 10) return fail(BEZ_ERR_UNSUPPORTED, "device %d is sm_%d%d; this build targets sm_103a", device,
                                     prop.major, prop.minor);
    bez_ctx c = new bez_ctx_s();
    c->device = device;
    c->sm_count = prop.multiProcessorCount;
    c->tex.max3d = prop.maxTexture3D[0] < prop.maxTexture3D[1] ? prop.maxTexture3D[0] : prop.maxTexture3D[1];
    c->tex.max2d_w = prop.maxTexture2D[0];
    c->tex.max2d_h = prop.maxTexture2D[1];
    BEZ_CUDA(cudaEventCreateWithFlags(&c->tex_done, cudaEventDisableTiming), "cudaEventCreate");
    *out = c;
    return BEZ_OK;
}

bez_status bez_destroy(bez_ctx c)
{
    if (!c) return BEZ_OK;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto& pr : c->pending) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto e : c->spare) cudaEventDestroy(e);
    for (auto& b : c->stage)
        if (b.p) cudaFree(b.p);
    atlas_free(c->tex.dc3);
    atlas_free(c->tex.strip2);
    atlas_free(c->tex.seil2);
    atlas_free(c->tex.seil2s);
    atlas_free(c->tex.seil3);
    atlas_free(c->tex.chain);
    atlas_free(c->tex.chain3);
    atlas_free(c->tex.probe);
    atlas_free(c->tex.probe2);
    atlas_free(c->tex.surf3);
    if (c->pipe_in) cudaStreamDestroy(c->pipe_in);
    if (c->pipe_out) cudaStreamDestroy(c->pipe_out);
    if (c->pipe_alt) cudaStreamDestroy(c->pipe_alt);
    for (auto e : c->pipe_ev)
        if (e) cudaEventDestroy(e);
    atlas_free(c->tex.surf2);
    cudaFree(c->tex.rescale);
    if (c->tex_done) cudaEventDestroy(c->tex_done);
    delete c;
    return BEZ_OK;
}

bez_status bez_set_timing(bez_ctx c, int enable)
{
    if (!c) return fail(BEZ_ERR_INVALID_ARG, "null context");
    c->timing = enable != 0;
    return BEZ_OK;
}

bez_status bez_get_stats(bez_ctx c, bez_stats* out)
{
    if (!c || !out) return fail(BEZ_ERR_INVALID_ARG, "null argument");
    for (auto& pr : c->pending) {
        BEZ_CUDA(cudaEventSynchronize(pr.second), "cudaEventSynchronize");
        float ms = 0.f;
        BEZ_CUDA(cudaEventElapsedTime(&ms, pr.first, pr.second), "cudaEventElapsedTime");
        c->timed_ms += ms;
        c->timed_launches += 1;
        c->spare.push_back(pr.first);
        c->spare.push_back(pr.second);
    }
    c->pending.clear();
    out->launches = c->launches;
    out->timed_launches = c->timed_launches;
    out->timed_ms = c->timed_ms;
    return BEZ_OK;
}

bez_status bez_reset_stats(bez_ctx c)
{
    bez_stats tmp;
    bez_status st = bez_get_stats(c, &tmp);
    if (st != BEZ_OK) return st;
    c->launches = 0;
    c->timed_launches = 0;
    c->timed_ms = 0.0;
    return BEZ_OK;
}

bez_status bez_eval(bez_ctx c, const void* ctrl, int64_t n_curves, int degree, int dim, const float* t, int64_t n_t,
                    float* out, const bez_opts* o, void* stream)
{
    bez_status st = check_common(c, o);
    if (st != BEZ_OK) return st;
    if (n_curves < 0 || n_t < 0) return fail(BEZ_ERR_INVALID_ARG, "negative size");
    if (n_t > 0x7fffffff) return fail(BEZ_ERR_INVALID_ARG, "n_t %lld exceeds 2^31-1", (long long)n_t);
    if (o->t_mode == BEZ_T_HASH && n_curves > 0xffffffffLL)
        return fail(BEZ_ERR_INVALID_ARG, "hash parameters index curves with 32 bits");
    if (dim < 1 || dim > 4) return fail(BEZ_ERR_INVALID_ARG, "dim %d not in 1..4", dim);
    if (degree < 1) return fail(BEZ_ERR_INVALID_ARG, "degree %d < 1", degree);
    // AUTO: the fastest register form within 1e-6 of the curve's extent up
    // to degree 7 (centred Horner), Seiler above
    int var = o->variant != BEZ_VAR_AUTO ? o->variant : degree <= 7 ? BEZ_VAR_HORNER_CENTRED : BEZ_VAR_SEILER;
    const bool coissue = var == BEZ_VAR_COISSUE;
    const bool tex = var == BEZ_VAR_TEX_DECASTELJAU || var == BEZ_VAR_TEX_SEILER || var == BEZ_VAR_TEX_HYBRID ||
                     coissue;
    const bool half2 = var == BEZ_VAR_HALF2;
    if (var > BEZ_VAR_TEX_HYBRID && !coissue && !half2)
        return fail(BEZ_ERR_UNSUPPORTED, "variant %d not available for bez_eval", var);
    if (half2 && (dim != 3 || degree > 7))
        return fail(BEZ_ERR_UNSUPPORTED, "half2 arithmetic evaluates 3D curves of degree 1..7");
    if (coissue) {
        if (degree != 3 || dim != 3 || o->out_mode != BEZ_OUT_POLYLINE_LENGTH || o->t_mode != BEZ_T_HASH ||
            n_t > 65536)
            return fail(BEZ_ERR_UNSUPPORTED,
                        "co-issue evaluates cubic 3D curves to polyline lengths at <= 65536 hashed parameters");
        if (o->tex_share < 0 || o->tex_share > 7)
            return fail(BEZ_ERR_INVALID_ARG, "tex_share %d not in 0..7", o->tex_share);
    }
    if (degree > kMaxDegree) return fail(BEZ_ERR_UNSUPPORTED, "degree %d > %d", degree, kMaxDegree);
    if (var == BEZ_VAR_TEX_SEILER && (degree < 2 || degree > 7))
        return fail(BEZ_ERR_UNSUPPORTED, "Seiler textures are defined for degrees 2..7 (got %d)", degree);
    if (o->tex_spread > 1 && !(var == BEZ_VAR_TEX_SEILER && degree <= 3))
        return fail(BEZ_ERR_UNSUPPORTED, "spread tiles (tex_spread %d) are built for TEX_SEILER of degree 2, 3",
                    o->tex_spread);
    if (tex && o->dtype == BEZ_BF16) return fail(BEZ_ERR_UNSUPPORTED, "no bfloat16 texture format");
    if (n_curves == 0 || (n_t == 0 && o->out_mode == BEZ_OUT_POINTS)) return BEZ_OK;
    if (!ctrl || !out) return fail(BEZ_ERR_INVALID_ARG, "null ctrl or out");
    const bool t_array = o->t_mode == BEZ_T_SHARED || o->t_mode == BEZ_T_PER_CURVE;
    if (t_array && n_t > 0 && !t) return fail(BEZ_ERR_INVALID_ARG, "null t for t_mode %d", o->t_mode);

    std::lock_guard<std::mutex> g(c->mu);
    BEZ_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Staging stg{c, s};
    CurveArgs a{};
    const size_t ctrl_per = (size_t)(degree + 1) * dim * dtype_size(o->dtype);
    const size_t ctrl_bytes = (size_t)n_curves * ctrl_per;
    // Host control points and host output on a register evaluator: run the
    // call as chunks whose copies in and out overlap the evaluation of the
    // neighbouring chunks (per-curve host parameters disable it).
    const bool pipe = !tex && classify(ctrl) == MEM_HOST && classify(out) == MEM_HOST &&
                      n_curves >= 2 * kPipeMinCurves && !(o->t_mode == BEZ_T_PER_CURVE && classify(t) == MEM_HOST);
    if (pipe) {
        st = ensure_stage(c, 0, ctrl_bytes, s);
        if (st != BEZ_OK) return st;
        a.ctrl = c->stage[0].p;
    } else {
        st = stg.in(ctrl, ctrl_bytes, 0, &a.ctrl);
        if (st != BEZ_OK) return st;
    }
    if (t_array) {
        const size_t tb = (size_t)n_t * sizeof(float) * (o->t_mode == BEZ_T_PER_CURVE ? (size_t)n_curves : 1);
        const void* td = nullptr;
        st = stg.in(t, tb, 1, &td);
        if (st != BEZ_OK) return st;
        a.t = static_cast<const float*>(td);
        a.t_stride = o->t_mode == BEZ_T_PER_CURVE ? n_t : 0;
    }
    const size_t out_per = o->out_mode == BEZ_OUT_POINTS ? (size_t)n_t * dim * sizeof(float) : sizeof(float);
    const size_t out_bytes = (size_t)n_curves * out_per;
    void* od = nullptr;
    if (pipe) {
        st = ensure_stage(c, 2, out_bytes, s);
        if (st != BEZ_OK) return st;
        od = c->stage[2].p;
    } else {
        st = stg.out(out, out_bytes, 2, &od);
        if (st != BEZ_OK) return st;
    }
    a.out = static_cast<float*>(od);
    a.dtype = o->dtype;
    a.degree = degree;
    a.dim = dim;
    a.n_t = (int32_t)n_t;
    a.n_curves = n_curves;
    const uint32_t seed_lo = (uint32_t)(o->seed & 0xffffffffu), seed_hi = (uint32_t)(o->seed >> 32);
    a.key = lowbias32(seed_lo ^ lowbias32(seed_hi ^ lowbias32(o->stream_id)));
    const int tm = t_array ? TM_ARRAY : (o->t_mode == BEZ_T_UNIFORM ? TM_UNIFORM : TM_HASH);
    const int om = o->out_mode == BEZ_OUT_POINTS ? OM_POINTS : OM_LENGTH;

    LaunchHooks h = hooks_of(c);
    LaunchResult r{0, cudaSuccess};
    if (tex) {
        // the atlases are shared by all calls of this context: order their use
        if (c->tex_used) BEZ_CUDA(cudaStreamWaitEvent(s, c->tex_done, 0), "cudaStreamWaitEvent");
        r = coissue ? launch_tex_coissue(a, o->tex_share ? o->tex_share : kDefaultTexShare, o->tex_format, c->tex, s, h)
                    : launch_tex_curve(a, var, tm, om, o->tex_format, o->tex_spread, c->tex, s, h);
        if (r.err == cudaErrorInvalidValue && r.launches == 0)
            return fail(BEZ_ERR_UNSUPPORTED, "batch of %lld curves does not fit one texture atlas",
                        (long long)n_curves);
        if (r.err != cudaSuccess) return cuda_fail(r.err, "texture evaluator");
        BEZ_CUDA(cudaEventRecord(c->tex_done, s), "cudaEventRecord");
        c->tex_used = true;
        return stg.finish(o->sync);
    }
    auto launch = [&](const CurveArgs& ak, cudaStream_t cs) {
        switch (var) {
        case BEZ_VAR_HORNER: return launch_curve_horner(ak, tm, om, cs, h);
        case BEZ_VAR_HORNER_CENTRED: return launch_curve_horner_centred(ak, tm, om, cs, h);
        case BEZ_VAR_BERNSTEIN: return launch_curve_bernstein(ak, tm, om, cs, h);
        case BEZ_VAR_DECASTELJAU: return launch_curve_decasteljau(ak, tm, om, cs, h);
        case BEZ_VAR_HALF2: return launch_curve_half2(ak, tm, om, cs, h);
        default: return launch_curve_seiler(ak, tm, om, cs, h);
        }
    };
    if (!pipe) {
        r = launch(a, s);
        if (r.err != cudaSuccess) return cuda_fail(r.err, "curve evaluator launch");
        return stg.finish(o->sync);
    }
    // chunk k: copy in on pipe_in, evaluate on s (even k) or pipe_alt (odd k),
    // copy out on pipe_out.  Alternating the evaluation streams lets chunk k + 1
    // take the SMs that chunk k's last wave leaves idle.
    if (!c->pipe_in) {
        BEZ_CUDA(cudaStreamCreateWithFlags(&c->pipe_in, cudaStreamNonBlocking), "cudaStreamCreate");
        BEZ_CUDA(cudaStreamCreateWithFlags(&c->pipe_out, cudaStreamNonBlocking), "cudaStreamCreate");
        BEZ_CUDA(cudaStreamCreateWithFlags(&c->pipe_alt, cudaStreamNonBlocking), "cudaStreamCreate");
        for (auto& e : c->pipe_ev) BEZ_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
    }
    const int K = (int)std::min<int64_t>(kPipeChunks, n_curves / kPipeMinCurves);
    cudaEvent_t* ev = c->pipe_ev;
    BEZ_CUDA(cudaEventRecord(ev[0], s), "cudaEventRecord");  // earlier work on s (e.g. the staged t) comes first
    BEZ_CUDA(cudaStreamWaitEvent(c->pipe_in, ev[0], 0), "cudaStreamWaitEvent");
    BEZ_CUDA(cudaStreamWaitEvent(c->pipe_out, ev[0], 0), "cudaStreamWaitEvent");
    BEZ_CUDA(cudaStreamWaitEvent(c->pipe_alt, ev[0], 0), "cudaStreamWaitEvent");
    const char* hin = static_cast<const char*>(ctrl);
    char* hout = reinterpret_cast<char*>(out);
    char* din = static_cast<char*>(c->stage[0].p);
    char* dout = static_cast<char*>(c->stage[2].p);
    // a short first chunk (1/32 of the curves) starts the evaluation early;
    // the rest is split evenly
    const int64_t head = n_curves / 32;
    auto bound = [&](int i) -> int64_t {
        return i == 0 ? 0 : i == K ? n_curves : head + (n_curves - head) * (i - 1) / (K - 1);
    };
    for (int k = 0; k < K; ++k) {
        const int64_t c0 = bound(k), c1 = bound(k + 1), nk = c1 - c0;
        BEZ_CUDA(cudaMemcpyAsync(din + c0 * ctrl_per, hin + c0 * ctrl_per, nk * ctrl_per, cudaMemcpyHostToDevice,
                                 c->pipe_in), "copy input chunk to device");
        BEZ_CUDA(cudaEventRecord(ev[1 + k], c->pipe_in), "cudaEventRecord");
        cudaStream_t cs = (k & 1) ? c->pipe_alt : s;
        BEZ_CUDA(cudaStreamWaitEvent(cs, ev[1 + k], 0), "cudaStreamWaitEvent");
        CurveArgs ak = a;
        ak.ctrl = din + c0 * ctrl_per;
        ak.out = reinterpret_cast<float*>(dout + c0 * out_per);
        ak.n_curves = nk;
        ak.c_base = c0;
        r = launch(ak, cs);
        if (r.err != cudaSuccess) return cuda_fail(r.err, "curve evaluator launch");
        BEZ_CUDA(cudaEventRecord(ev[1 + kPipeChunks + k], cs), "cudaEventRecord");
        BEZ_CUDA(cudaStreamWaitEvent(c->pipe_out, ev[1 + kPipeChunks + k], 0), "cudaStreamWaitEvent");
        BEZ_CUDA(cudaMemcpyAsync(hout + c0 * out_per, dout + c0 * out_per, nk * out_per, cudaMemcpyDeviceToHost,
                                 c->pipe_out), "copy output chunk to host");
    }
    BEZ_CUDA(cudaEventRecord(ev[1 + 2 * kPipeChunks], c->pipe_out), "cudaEventRecord");
    BEZ_CUDA(cudaStreamWaitEvent(s, ev[1 + 2 * kPipeChunks], 0), "cudaStreamWaitEvent");
    BEZ_CUDA(cudaStreamSynchronize(s), "stream synchronize");
    return BEZ_OK;
}

bez_status bez_eval_piecewise(bez_ctx c, const void* ctrl, int64_t n_chains, int n_seg, int degree, int dim,
                              const float* t, int64_t n_t, float* out, const bez_opts* o, void* stream)
{
    bez_status st = check_common(c, o);
    if (st != BEZ_OK) return st;
    if (n_chains < 0 || n_t < 0) return fail(BEZ_ERR_INVALID_ARG, "negative size");
    if (n_t > 0x7fffffff) return fail(BEZ_ERR_INVALID_ARG, "n_t %lld exceeds 2^31-1", (long long)n_t);
    if (o->t_mode == BEZ_T_HASH && n_chains > 0xffffffffLL)
        return fail(BEZ_ERR_INVALID_ARG, "hash parameters index chains with 32 bits");
    if (dim < 1 || dim > 4) return fail(BEZ_ERR_INVALID_ARG, "dim %d not in 1..4", dim);
    if (degree < 1 || n_seg < 1) return fail(BEZ_ERR_INVALID_ARG, "degree %d / n_seg %d must be >= 1", degree, n_seg);
    int var = o->variant == BEZ_VAR_AUTO ? BEZ_VAR_DECASTELJAU : o->variant;
    const bool tex = var == BEZ_VAR_TEX_DECASTELJAU;
    if (var > BEZ_VAR_TEX_DECASTELJAU || var == BEZ_VAR_TENSOR)
        return fail(BEZ_ERR_UNSUPPORTED, "variant %d not available for chains", var);
    if (tex && degree != 2 && degree != 3)
        return fail(BEZ_ERR_UNSUPPORTED, "zig-zag chain textures hold quadratic or cubic segments (degree %d)",
                    degree);
    if (tex && degree == 3 && o->tex_spread > 1)
        return fail(BEZ_ERR_UNSUPPORTED, "cubic zig-zag chains use the (N+1) x 2 x 2 layout (tex_spread 0 or 1)");
    if (tex && o->dtype == BEZ_BF16) return fail(BEZ_ERR_UNSUPPORTED, "no bfloat16 texture format");
    if (tex && o->tex_format == BEZ_TEX_UNORM8)
        return fail(BEZ_ERR_UNSUPPORTED, "zig-zag texels span tens of the control points' extent: unorm8 is too coarse");
    if (tex && o->tex_format == BEZ_TEX_UNORM16 && (degree != 2 || o->dtype != BEZ_F32))
        return fail(BEZ_ERR_UNSUPPORTED, "unorm16 chain textures: quadratic chains of FP32 control points");
    if (!tex && o->tex_spread > 1)
        return fail(BEZ_ERR_UNSUPPORTED, "tex_spread applies to the zig-zag chain texture (TEX_DECASTELJAU)");
    if (degree > kMaxDegree) return fail(BEZ_ERR_UNSUPPORTED, "degree %d > %d", degree, kMaxDegree);
    const int64_t per = ((int64_t)n_seg * degree + 1) * dim;
    if (!tex && per > kChainMaxFloats)
        return fail(BEZ_ERR_UNSUPPORTED, "chain of %lld control values exceeds %d", (long long)per, kChainMaxFloats);
    if (n_chains == 0 || (n_t == 0 && o->out_mode == BEZ_OUT_POINTS)) return BEZ_OK;
    if (!ctrl || !out) return fail(BEZ_ERR_INVALID_ARG, "null ctrl or out");
    const bool t_array = o->t_mode == BEZ_T_SHARED || o->t_mode == BEZ_T_PER_CURVE;
    if (t_array && n_t > 0 && !t) return fail(BEZ_ERR_INVALID_ARG, "null t for t_mode %d", o->t_mode);

    std::lock_guard<std::mutex> g(c->mu);
    BEZ_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Staging stg{c, s};
    CurveArgs a{};
    st = stg.in(ctrl, (size_t)n_chains * per * dtype_size(o->dtype), 0, &a.ctrl);
    if (st != BEZ_OK) return st;
    if (t_array) {
        const size_t tb = (size_t)n_t * sizeof(float) * (o->t_mode == BEZ_T_PER_CURVE ? (size_t)n_chains : 1);
        const void* td = nullptr;
        st = stg.in(t, tb, 1, &td);
        if (st != BEZ_OK) return st;
        a.t = static_cast<const float*>(td);
        a.t_stride = o->t_mode == BEZ_T_PER_CURVE ? n_t : 0;
    }
    const size_t out_bytes =
        o->out_mode == BEZ_OUT_POINTS ? (size_t)n_chains * n_t * dim * sizeof(float) : (size_t)n_chains * sizeof(float);
    void* od = nullptr;
    st = stg.out(out, out_bytes, 2, &od);
    if (st != BEZ_OK) return st;
    a.out = static_cast<float*>(od);
    a.dtype = o->dtype;
    a.degree = degree;
    a.dim = dim;
    a.n_t = (int32_t)n_t;
    a.n_curves = n_chains;
    a.n_seg = n_seg;
    const uint32_t seed_lo = (uint32_t)(o->seed & 0xffffffffu), seed_hi = (uint32_t)(o->seed >> 32);
    a.key = lowbias32(seed_lo ^ lowbias32(seed_hi ^ lowbias32(o->stream_id)));
    const int tm = t_array ? TM_ARRAY : (o->t_mode == BEZ_T_UNIFORM ? TM_UNIFORM : TM_HASH);
    const int om = o->out_mode == BEZ_OUT_POINTS ? OM_POINTS : OM_LENGTH;
    LaunchHooks h = hooks_of(c);
    LaunchResult r{0, cudaSuccess};
    if (tex) {
        if (c->tex_used) BEZ_CUDA(cudaStreamWaitEvent(s, c->tex_done, 0), "cudaStreamWaitEvent");
        r = launch_tex_chain(a, tm, om, o->tex_spread, o->tex_format, c->tex, s, h);
        if (r.err == cudaErrorInvalidValue && r.launches == 0)
            return fail(BEZ_ERR_UNSUPPORTED, "%lld chains of %d segments do not fit one texture atlas",
                        (long long)n_chains, n_seg);
        if (r.err != cudaSuccess) return cuda_fail(r.err, "zig-zag chain evaluator");
        BEZ_CUDA(cudaEventRecord(c->tex_done, s), "cudaEventRecord");
        c->tex_used = true;
        return stg.finish(o->sync);
    }
    switch (var) {
    case BEZ_VAR_HORNER: r = launch_chain_horner(a, tm, om, s, h); break;
    case BEZ_VAR_HORNER_CENTRED: r = launch_chain_horner_centred(a, tm, om, s, h); break;
    case BEZ_VAR_BERNSTEIN: r = launch_chain_bernstein(a, tm, om, s, h); break;
    case BEZ_VAR_SEILER: r = launch_chain_seiler(a, tm, om, s, h); break;
    default: r = launch_chain_decasteljau(a, tm, om, s, h); break;
    }
    if (r.err != cudaSuccess) return cuda_fail(r.err, "chain evaluator launch");
    return stg.finish(o->sync);
}

static bez_status eval_spline(bez_ctx c, const float* ctrl, const float* weights, const float* knots, int64_t n_curves,
                              int n_ctrl, int degree, int dim, const float* t, int64_t n_t, float* out,
                              const bez_opts* o, void* stream, bool rational)
{
    bez_status st = check_common(c, o);
    if (st != BEZ_OK) return st;
    if (n_curves < 0 || n_t < 0) return fail(BEZ_ERR_INVALID_ARG, "negative size");
    if (n_t > 0x7fffffff) return fail(BEZ_ERR_INVALID_ARG, "n_t %lld exceeds 2^31-1", (long long)n_t);
    if (o->t_mode == BEZ_T_HASH && n_curves > 0xffffffffLL)
        return fail(BEZ_ERR_INVALID_ARG, "hash parameters index curves with 32 bits");
    if (dim < 1 || dim > 4) return fail(BEZ_ERR_INVALID_ARG, "dim %d not in 1..4", dim);
    if (degree < 1 || n_ctrl < degree + 1)
        return fail(BEZ_ERR_INVALID_ARG, "need degree >= 1 and n_ctrl >= degree+1 (degree %d, n_ctrl %d)", degree,
                    n_ctrl);
    if (degree > kMaxDegree) return fail(BEZ_ERR_UNSUPPORTED, "degree %d > %d", degree, kMaxDegree);
    if (o->dtype != BEZ_F32) return fail(BEZ_ERR_UNSUPPORTED, "splines take FP32 control points");
    const int var = o->variant == BEZ_VAR_AUTO ? BEZ_VAR_DECASTELJAU : o->variant;
    if (var != BEZ_VAR_DECASTELJAU)
        return fail(BEZ_ERR_UNSUPPORTED, "splines evaluate their Bezier spans by de Casteljau (variant %d)", var);
    if (rational && !weights && n_curves > 0) return fail(BEZ_ERR_INVALID_ARG, "null weights");
    if (n_curves == 0 || (n_t == 0 && o->out_mode == BEZ_OUT_POINTS)) return BEZ_OK;
    if (!ctrl || !out) return fail(BEZ_ERR_INVALID_ARG, "null ctrl or out");
    const bool t_array = o->t_mode == BEZ_T_SHARED || o->t_mode == BEZ_T_PER_CURVE;
    if (t_array && n_t > 0 && !t) return fail(BEZ_ERR_INVALID_ARG, "null t for t_mode %d", o->t_mode);

    std::lock_guard<std::mutex> g(c->mu);
    BEZ_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Staging stg{c, s};
    SplineArgs a{};
    const void* p = nullptr;
    st = stg.in(ctrl, (size_t)n_curves * n_ctrl * dim * sizeof(float), 0, &p);
    if (st != BEZ_OK) return st;
    a.ctrl = static_cast<const float*>(p);
    if (rational) {
        st = stg.in(weights, (size_t)n_curves * n_ctrl * sizeof(float), 3, &p);
        if (st != BEZ_OK) return st;
        a.weights = static_cast<const float*>(p);
    }
    if (knots) {
        st = stg.in(knots, (size_t)n_curves * (n_ctrl + degree + 1) * sizeof(float), 4, &p);
        if (st != BEZ_OK) return st;
        a.knots = static_cast<const float*>(p);
    }
    if (t_array) {
        const size_t tb = (size_t)n_t * sizeof(float) * (o->t_mode == BEZ_T_PER_CURVE ? (size_t)n_curves : 1);
        st = stg.in(t, tb, 1, &p);
        if (st != BEZ_OK) return st;
        a.t = static_cast<const float*>(p);
        a.t_stride = o->t_mode == BEZ_T_PER_CURVE ? n_t : 0;
    }
    const size_t out_bytes =
        o->out_mode == BEZ_OUT_POINTS ? (size_t)n_curves * n_t * dim * sizeof(float) : (size_t)n_curves * sizeof(float);
    void* od = nullptr;
    st = stg.out(out, out_bytes, 2, &od);
    if (st != BEZ_OK) return st;
    a.out = static_cast<float*>(od);
    a.n_curves = n_curves;
    a.n_ctrl = n_ctrl;
    a.degree = degree;
    a.dim = dim;
    a.comps = rational ? dim + 1 : dim;
    a.n_spans = n_ctrl - degree;
    a.n_t = (int32_t)n_t;
    a.err_word = o->err_word;
    const uint32_t seed_lo = (uint32_t)(o->seed & 0xffffffffu), seed_hi = (uint32_t)(o->seed >> 32);
    a.key = lowbias32(seed_lo ^ lowbias32(seed_hi ^ lowbias32(o->stream_id)));
    // Bezier spans: library-owned scratch, one slot per context
    const size_t span_bytes = (size_t)n_curves * a.n_spans * (degree + 1) * a.comps * sizeof(float);
    st = ensure_stage(c, 5, span_bytes, s);
    if (st != BEZ_OK) return st;
    a.spans = static_cast<float*>(c->stage[5].p);
    const int tm = t_array ? TM_ARRAY : (o->t_mode == BEZ_T_UNIFORM ? TM_UNIFORM : TM_HASH);
    const int om = o->out_mode == BEZ_OUT_POINTS ? OM_POINTS : OM_LENGTH;
    LaunchHooks h = hooks_of(c);
    LaunchResult r = launch_spline_setup(a, s, h);
    if (r.err != cudaSuccess) return cuda_fail(r.err, "spline setup launch");
    r = launch_spline_eval(a, tm, om, s, h);
    if (r.err != cudaSuccess) return cuda_fail(r.err, "spline evaluator launch");
    return stg.finish(o->sync);
}

bez_status bez_eval_bspline(bez_ctx c, const float* ctrl, const float* knots, int64_t n_curves, int n_ctrl,
                            int degree, int dim, const float* t, int64_t n_t, float* out, const bez_opts* o,
                            void* stream)
{
    return eval_spline(c, ctrl, nullptr, knots, n_curves, n_ctrl, degree, dim, t, n_t, out, o, stream, false);
}

bez_status bez_eval_nurbs(bez_ctx c, const float* ctrl, const float* weights, const float* knots, int64_t n_curves,
                          int n_ctrl, int degree, int dim, const float* t, int64_t n_t, float* out,
                          const bez_opts* o, void* stream)
{
    return eval_spline(c, ctrl, weights, knots, n_curves, n_ctrl, degree, dim, t, n_t, out, o, stream, true);
}

static bez_status eval_tensor(bez_ctx c, const void* ctrl, int64_t n, int du, int dv, int dw, int dim, int nu, int nv,
                              int nw, float* out, const bez_opts* o, void* stream)
{
    bez_status st = check_common(c, o);
    if (st != BEZ_OK) return st;
    const bool vol = dw >= 0;
    if (n < 0) return fail(BEZ_ERR_INVALID_ARG, "negative size");
    if (dim < 1 || dim > 4) return fail(BEZ_ERR_INVALID_ARG, "dim %d not in 1..4", dim);
    if (du < 1 || dv < 1 || (vol && dw < 1)) return fail(BEZ_ERR_INVALID_ARG, "degrees must be >= 1");
    if (nu < 1 || nv < 1 || (vol && nw < 1)) return fail(BEZ_ERR_INVALID_ARG, "grid sizes must be >= 1");
    if (du > 7 || dv > 7 || dw > 7) return fail(BEZ_ERR_UNSUPPORTED, "tensor-product degrees above 7");
    if (nu > 256 || nv > 256 || nw > 256) return fail(BEZ_ERR_UNSUPPORTED, "grids above 256 per axis");
    if (o->out_mode != BEZ_OUT_POINTS) return fail(BEZ_ERR_UNSUPPORTED, "surfaces and volumes output points");
    const int var = o->variant;
    const bool tex = var == BEZ_VAR_TEX_DECASTELJAU || var == BEZ_VAR_TEX_SEILER;
    if (var != BEZ_VAR_AUTO && var != BEZ_VAR_BERNSTEIN && !tex)
        return fail(BEZ_ERR_UNSUPPORTED,
                    "variant %d: grids run on CUDA cores (AUTO / BERNSTEIN) or, for bicubic surfaces and tricubic "
                    "scalar volumes, through texture tiles (TEX_DECASTELJAU, TEX_SEILER)", var);
    if (tex && (du != 3 || dv != 3 || (vol && (dw != 3 || dim != 1))))
        return fail(BEZ_ERR_UNSUPPORTED, "texture tiles hold bicubic surfaces and tricubic scalar volumes only");
    if (tex && !vol && nu > kSurfTexMaxRows)
        return fail(BEZ_ERR_UNSUPPORTED, "texture surfaces take at most %d rows in u", kSurfTexMaxRows);
    if (tex && vol && (nu > kVolTexMaxRows || nw % 4 != 0))
        return fail(BEZ_ERR_UNSUPPORTED, "texture volumes take at most %d rows in u and nw a multiple of 4",
                    kVolTexMaxRows);
    if (tex && o->dtype == BEZ_BF16) return fail(BEZ_ERR_UNSUPPORTED, "no bfloat16 texture format");
    if (o->tex_spread > 1 && var != BEZ_VAR_TEX_SEILER)
        return fail(BEZ_ERR_UNSUPPORTED, "spread tiles are built for TEX_SEILER surfaces and volumes");
    TensorLaunch t{};
    t.dtype = o->dtype;
    t.n = n;
    t.du = du;
    t.dv = dv;
    t.dw = vol ? dw : -1;
    t.dim = dim;
    t.nu = nu;
    t.nv = nv;
    t.nw = vol ? nw : 1;
    if (tensor_product_smem(t) > 200 * 1024) return fail(BEZ_ERR_UNSUPPORTED, "grid too large for one block");
    if (n == 0) return BEZ_OK;
    if (!ctrl || !out) return fail(BEZ_ERR_INVALID_ARG, "null ctrl or out");
    std::lock_guard<std::mutex> g(c->mu);
    BEZ_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Staging stg{c, s};
    const int64_t per = (int64_t)(du + 1) * (dv + 1) * (vol ? dw + 1 : 1) * dim;
    st = stg.in(ctrl, (size_t)n * per * dtype_size(o->dtype), 0, &t.ctrl);
    if (st != BEZ_OK) return st;
    void* od = nullptr;
    st = stg.out(out, (size_t)n * nu * nv * (vol ? nw : 1) * dim * sizeof(float), 2, &od);
    if (st != BEZ_OK) return st;
    t.out = static_cast<float*>(od);
    if (tex && vol && (reinterpret_cast<uintptr_t>(t.out) & 15) != 0)
        return fail(BEZ_ERR_UNSUPPORTED, "texture volumes write float4s: out must be 16-byte aligned");
    if (tex) {
        // the atlases are shared by all calls of this context: order their use
        if (c->tex_used) BEZ_CUDA(cudaStreamWaitEvent(s, c->tex_done, 0), "cudaStreamWaitEvent");
        LaunchResult r =
            launch_tex_surface(t, var == BEZ_VAR_TEX_SEILER, o->tex_format, o->tex_spread, c->tex, s, hooks_of(c));
        if (r.err == cudaErrorInvalidValue && r.launches == 0)
            return fail(BEZ_ERR_UNSUPPORTED, "%lld patches do not fit one texture atlas", (long long)n);
        if (r.err != cudaSuccess) return cuda_fail(r.err, "texture tile launch");
        BEZ_CUDA(cudaEventRecord(c->tex_done, s), "cudaEventRecord");
        c->tex_used = true;
        return stg.finish(o->sync);
    }
    LaunchResult r = launch_tensor_product(t, s, hooks_of(c));
    if (r.err != cudaSuccess) return cuda_fail(r.err, "tensor-product launch");
    return stg.finish(o->sync);
}

bez_status bez_eval_surface(bez_ctx c, const void* ctrl, int64_t n, int du, int dv, int dim, int nu, int nv,
                            float* out, const bez_opts* o, void* stream)
{
    return eval_tensor(c, ctrl, n, du, dv, -1, dim, nu, nv, 1, out, o, stream);
}

bez_status bez_eval_volume(bez_ctx c, const void* ctrl, int64_t n, int du, int dv, int dw, int dim, int nu, int nv,
                           int nw, float* out, const bez_opts* o, void* stream)
{
    if (dw < 0) return fail(BEZ_ERR_INVALID_ARG, "degree %d < 1", dw);
    return eval_tensor(c, ctrl, n, du, dv, dw, dim, nu, nv, nw, out, o, stream);
}

// The adjoint, with an upstream gradient (grad_out) or the fused squared
// error against targets (target, loss_scale, loss).
static bez_status adjoint(bez_ctx c, const float* ctrl, const float* weights, int64_t n_curves, int degree, int dim,
                          const float* t, int64_t n_t, const float* grad_out, const float* target, float loss_scale,
                          float* loss, float* grad_ctrl, float* grad_weights, float* grad_t, const bez_opts* o,
                          void* stream)
{
    bez_status st = check_common(c, o);
    if (st != BEZ_OK) return st;
    if (n_curves < 0 || n_t < 0) return fail(BEZ_ERR_INVALID_ARG, "negative size");
    if (n_t > 0x7fffffff) return fail(BEZ_ERR_INVALID_ARG, "n_t %lld exceeds 2^31-1", (long long)n_t);
    if (dim < 1 || dim > 4) return fail(BEZ_ERR_INVALID_ARG, "dim %d not in 1..4", dim);
    if (degree < 1) return fail(BEZ_ERR_INVALID_ARG, "degree %d < 1", degree);
    if (degree > kMaxDegree) return fail(BEZ_ERR_UNSUPPORTED, "degree %d > %d", degree, kMaxDegree);
    if (o->dtype != BEZ_F32) return fail(BEZ_ERR_UNSUPPORTED, "the adjoint takes FP32 control points");
    if (o->t_mode != BEZ_T_SHARED && o->t_mode != BEZ_T_PER_CURVE)
        return fail(BEZ_ERR_UNSUPPORTED, "the adjoint needs the parameters as an array (SHARED / PER_CURVE)");
    if (grad_weights && !weights) return fail(BEZ_ERR_INVALID_ARG, "grad_weights requested without weights");
    if (n_curves == 0) return BEZ_OK;
    if (!ctrl || (n_t > 0 && (!t || (!grad_out && !target))))
        return fail(BEZ_ERR_INVALID_ARG, "null ctrl, t, grad_out or target");
    std::lock_guard<std::mutex> g(c->mu);
    BEZ_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Staging stg{c, s};
    GradArgs a{};
    const bool per_curve = o->t_mode == BEZ_T_PER_CURVE;
    const void* p = nullptr;
    st = stg.in(ctrl, (size_t)n_curves * (degree + 1) * dim * sizeof(float), 0, &p);
    if (st != BEZ_OK) return st;
    a.ctrl = static_cast<const float*>(p);
    if (weights) {
        st = stg.in(weights, (size_t)n_curves * (degree + 1) * sizeof(float), 3, &p);
        if (st != BEZ_OK) return st;
        a.weights = static_cast<const float*>(p);
    }
    st = stg.in(t, (size_t)n_t * sizeof(float) * (per_curve ? (size_t)n_curves : 1), 1, &p);
    if (st != BEZ_OK) return st;
    a.t = static_cast<const float*>(p);
    st = stg.in(target ? target : grad_out, (size_t)n_curves * n_t * dim * sizeof(float), 4, &p);
    if (st != BEZ_OK) return st;
    if (target) {
        a.target = static_cast<const float*>(p);
        a.loss_scale = loss_scale;
    } else {
        a.g = static_cast<const float*>(p);
    }
    void* od = nullptr;
    if (loss) {
        st = stg.out(loss, (size_t)n_curves * sizeof(float), 8, &od);
        if (st != BEZ_OK) return st;
        a.loss = static_cast<float*>(od);
    }
    if (grad_ctrl) {
        st = stg.out(grad_ctrl, (size_t)n_curves * (degree + 1) * dim * sizeof(float), 2, &od);
        if (st != BEZ_OK) return st;
        a.grad_ctrl = static_cast<float*>(od);
    }
    if (grad_weights) {
        st = stg.out(grad_weights, (size_t)n_curves * (degree + 1) * sizeof(float), 6, &od);
        if (st != BEZ_OK) return st;
        a.grad_w = static_cast<float*>(od);
    }
    if (grad_t) {
        const size_t gb = (size_t)n_t * sizeof(float) * (per_curve ? (size_t)n_curves : 1);
        st = stg.out(grad_t, gb, 7, &od);
        if (st != BEZ_OK) return st;
        a.grad_t = static_cast<float*>(od);
        if (!per_curve) BEZ_CUDA(cudaMemsetAsync(a.grad_t, 0, gb, s), "cudaMemsetAsync");
    }
    a.n_curves = n_curves;
    a.degree = degree;
    a.dim = dim;
    a.n_t = (int32_t)n_t;
    a.t_stride = per_curve ? n_t : 0;
    a.shared_gt = (!per_curve && n_t <= 8192) ? 1 : 0;
    LaunchResult r = launch_grad(a, s, hooks_of(c));
    if (r.err != cudaSuccess) return cuda_fail(r.err, "adjoint launch");
    return stg.finish(o->sync);
}

bez_status bez_eval_backward(bez_ctx c, const float* ctrl, const float* weights, int64_t n_curves, int degree, int dim,
                             const float* t, int64_t n_t, const float* grad_out, float* grad_ctrl,
                             float* grad_weights, float* grad_t, const bez_opts* o, void* stream)
{
    return adjoint(c, ctrl, weights, n_curves, degree, dim, t, n_t, grad_out, nullptr, 0.f, nullptr, grad_ctrl,
                   grad_weights, grad_t, o, stream);
}

bez_status bez_mse_grad(bez_ctx c, const float* ctrl, const float* weights, int64_t n_curves, int degree, int dim,
                        const float* t, int64_t n_t, const float* target, float loss_scale, float* loss,
                        float* grad_ctrl, float* grad_weights, float* grad_t, const bez_opts* o, void* stream)
{
    if (n_t > 0 && n_curves > 0 && !target) return fail(BEZ_ERR_INVALID_ARG, "null target");
    return adjoint(c, ctrl, weights, n_curves, degree, dim, t, n_t, nullptr, target, loss_scale, loss, grad_ctrl,
                   grad_weights, grad_t, o, stream);
}

bez_status bez_measure_peak(bez_ctx c, int kind, double* value, void* stream)
{
    if (!c || !value) return fail(BEZ_ERR_INVALID_ARG, "null argument");
    if (kind < BEZ_PEAK_FMA || kind > BEZ_PEAK_COPY) return fail(BEZ_ERR_INVALID_ARG, "unknown peak kind %d", kind);
    std::lock_guard<std::mutex> g(c->mu);
    BEZ_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    *value = 0.0;
    BEZ_CUDA(measure_peak(kind, c->sm_count, static_cast<cudaStream_t>(stream), value), "peak microbenchmark");
    return BEZ_OK;
}

bez_status bez_probe_filter(bez_ctx c, const float* xyz, int64_t n, float* out, void* stream)
{
    if (!c) return fail(BEZ_ERR_INVALID_ARG, "null context");
    if (n < 0) return fail(BEZ_ERR_INVALID_ARG, "negative size");
    if (n > 0 && (!xyz || !out)) return fail(BEZ_ERR_INVALID_ARG, "null coordinates or output");
    std::lock_guard<std::mutex> g(c->mu);
    BEZ_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Staging stg{c, s};
    const void* xd = nullptr;
    void* od = nullptr;
    bez_status st = stg.in(xyz, (size_t)n * 3 * sizeof(float), 0, &xd);
    if (st != BEZ_OK) return st;
    st = stg.out(out, (size_t)n * 4 * sizeof(float), 2, &od);
    if (st != BEZ_OK) return st;
    if (c->tex_used) BEZ_CUDA(cudaStreamWaitEvent(s, c->tex_done, 0), "cudaStreamWaitEvent");
    LaunchResult r = launch_tex_probe(static_cast<const float*>(xd), n, static_cast<float*>(od), c->tex, s,
                                      hooks_of(c));
    if (r.err != cudaSuccess) return cuda_fail(r.err, "filter probe");
    BEZ_CUDA(cudaEventRecord(c->tex_done, s), "cudaEventRecord");
    c->tex_used = true;
    return stg.finish(1);
}

bez_status bez_probe_filter_2d(bez_ctx c, const float* xy, int64_t n, float* out, void* stream)
{
    if (!c) return fail(BEZ_ERR_INVALID_ARG, "null context");
    if (n < 0) return fail(BEZ_ERR_INVALID_ARG, "negative size");
    if (n > 0 && (!xy || !out)) return fail(BEZ_ERR_INVALID_ARG, "null coordinates or output");
    std::lock_guard<std::mutex> g(c->mu);
    BEZ_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Staging stg{c, s};
    const void* xd = nullptr;
    void* od = nullptr;
    bez_status st = stg.in(xy, (size_t)n * 2 * sizeof(float), 0, &xd);
    if (st != BEZ_OK) return st;
    st = stg.out(out, (size_t)n * 4 * sizeof(float), 2, &od);
    if (st != BEZ_OK) return st;
    if (c->tex_used) BEZ_CUDA(cudaStreamWaitEvent(s, c->tex_done, 0), "cudaStreamWaitEvent");
    LaunchResult r = launch_tex_probe2d(static_cast<const float*>(xd), n, static_cast<float*>(od), c->tex, s,
                                        hooks_of(c));
    if (r.err != cudaSuccess) return cuda_fail(r.err, "2D filter probe");
    BEZ_CUDA(cudaEventRecord(c->tex_done, s), "cudaEventRecord");
    c->tex_used = true;
    return stg.finish(1);
}

}  // extern "C"
