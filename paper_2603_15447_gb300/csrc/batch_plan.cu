// batch_plan.cu -- host side of mixed batches: descriptor validation, work
// items, plan-owned device buffers, the autotuner and CUDA-graph capture.
// Kernels are in batch.cu; the ABI is declared in include/bez.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "context.h"
#include "spline.cuh"

using namespace bez;

namespace {

struct Shape {
    int chunk = 512;
    int schedule = 0;
    int threads = 256;
    int repr = 1;  // 0 Bezier points + de Casteljau, 1 centred power basis + Horner
    int partition = 0;  // atomic schedule: classes share the GPU by measured work (grids set by tune_partition)
};

void no_count(void*) {}
void no_event(void*, cudaStream_t) {}

std::mutex g_tune_mu;
std::map<std::string, Shape> g_tune_cache;

// ---- the JSON autotune cache: {"key": {"chunk": c, "schedule": s, "threads": t}, ...}

void load_cache_file(const char* path)
{
    FILE* f = fopen(path, "r");
    if (!f) return;
    std::string s;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, n);
    fclose(f);
    size_t pos = 0;
    for (;;) {
        const size_t k0 = s.find('"', pos);
        if (k0 == std::string::npos) break;
        const size_t k1 = s.find('"', k0 + 1);
        if (k1 == std::string::npos) break;
        const std::string key = s.substr(k0 + 1, k1 - k0 - 1);
        const size_t b0 = s.find('{', k1), b1 = s.find('}', k1);
        if (b0 == std::string::npos || b1 == std::string::npos || b0 > b1) {
            pos = k1 + 1;
            continue;
        }
        const std::string body = s.substr(b0, b1 - b0);
        Shape sh;
        auto field = [&](const char* name, int* out) {
            const size_t p = body.find(name);
            if (p != std::string::npos) *out = atoi(body.c_str() + body.find(':', p) + 1);
        };
        field("\"chunk\"", &sh.chunk);
        field("\"schedule\"", &sh.schedule);
        field("\"threads\"", &sh.threads);
        field("\"repr\"", &sh.repr);
        field("\"partition\"", &sh.partition);
        if (sh.chunk > 0 && sh.chunk % 256 == 0 && (sh.schedule == 0 || sh.schedule == 1) &&
            (sh.threads == 128 || sh.threads == 256) && (sh.repr == 0 || sh.repr == 1) &&
            (sh.partition == 0 || (sh.partition == 1 && sh.schedule == 1)))
            g_tune_cache[key] = sh;
        pos = b1 + 1;
    }
}

void save_cache_file(const char* path)
{
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    size_t i = 0;
    for (auto& kv : g_tune_cache) {
        fprintf(f, "  \"%s\": {\"chunk\": %d, \"schedule\": %d, \"threads\": %d, \"repr\": %d, \"partition\": %d}%s\n",
                kv.first.c_str(), kv.second.chunk, kv.second.schedule, kv.second.threads, kv.second.repr,
                kv.second.partition, ++i < g_tune_cache.size() ? "," : "");
    }
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

int log2_bucket(double x) { return x < 1 ? 0 : (int)std::lround(std::log2(x)); }

}  // namespace

struct bez_batch_s {
    bez_ctx ctx = nullptr;
    BatchArgs a{};
    std::vector<bez_curve_desc> hdesc;
    bez_curve_desc* d_desc = nullptr;
    float2* d_ops = nullptr;    // span operators M (Bezier-point representation)
    float2* d_ops_c = nullptr;  // T_p M (centred power-basis representation)
    SpanRec* d_span_rec = nullptr;
    bool spans_ready = false;
    BatchItem* d_items = nullptr;
    size_t items_cap = 0;
    std::vector<int64_t> hspan_off;   // per curve, floats into the span pool
    BatchStreams streams{};
    bool have_streams = false;
    float* d_spans = nullptr;
    void* d_counter = nullptr;
    Shape shape;
    bool setup_each = true;
    bool use_graph = false;
    cudaGraphExec_t exec = nullptr;
    int kernels_per_launch = 0;
    std::string key;
};

namespace {

// T[m][i]: coefficient of Bezier point b_i in the power coefficient c_m about
// t = 1/2 (degree p), c_m = binom(p, m) * (Bernstein value at 1/2 of the m-th
// forward differences), by applying the conversion to unit vectors in FP64
// (entries are small integers over powers of two, exact in FP64).
void centred_matrix(int p, double (&T)[8][8])
{
    for (int i = 0; i <= p; ++i) {
        double w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        w[i] = 1.0;
        double bin = 1.0;
        for (int m = 0; m <= p; ++m) {
            double h[8];
            for (int k = 0; k <= p - m; ++k) h[k] = w[k];
            for (int r = 1; r <= p - m; ++r)
                for (int k = 0; k <= p - m - r; ++k) h[k] = 0.5 * (h[k] + h[k + 1]);
            T[m][i] = bin * h[0];
            bin = bin * (double)(p - m) / (double)(m + 1);
            for (int k = 0; k < p - m; ++k) w[k] = w[k + 1] - w[k];
        }
    }
}

const BatchStreams* streams_of(bez_batch b) { return b->have_streams ? &b->streams : nullptr; }

bez_status build_items(bez_batch b, int chunk, cudaStream_t s)
{
    // items grouped by class (one evaluator kernel per class)
    std::vector<std::vector<BatchItem>> per_class(kBatchClasses);
    for (size_t c = 0; c < b->hdesc.size(); ++c) {
        const bez_curve_desc& d = b->hdesc[c];
        const int n = d.n_samples;
        auto& v = per_class[batch_item_class(d, b->a.dim)];
        for (int k = 0; (int64_t)k * chunk < n; ++k) {
            BatchItem it{};
            it.j0 = k * chunk;
            it.j1 = (int)std::min<int64_t>((int64_t)(k + 1) * chunk, n);
            it.n_samples = n;
            it.n_spans = d.type == BEZ_CURVE_BEZIER ? 0 : d.n_ctrl - d.degree;
            it.degree = d.degree;
            it.rational = d.type == BEZ_CURVE_NURBS;
            it.out_off = d.out_off;
            it.span_base = b->hspan_off[c];
            v.push_back(it);
        }
    }
    // Within a class, longest items first (largest-processing-time order):
    // warps that take the short items last finish close together, so the
    // class kernel's last wave is short for either schedule.
    for (auto& v : per_class)
        std::stable_sort(v.begin(), v.end(),
                         [](const BatchItem& x, const BatchItem& y) { return x.j1 - x.j0 > y.j1 - y.j0; });
    std::vector<BatchItem> items;
    for (int k = 0; k < kBatchClasses; ++k) {
        b->a.class_start[k] = (int64_t)items.size();
        items.insert(items.end(), per_class[k].begin(), per_class[k].end());
    }
    for (int k = kBatchClasses; k < 16; ++k) b->a.class_start[k] = (int64_t)items.size();
    if (items.size() > b->items_cap) {
        if (b->d_items) {
            cudaError_t e = cudaStreamSynchronize(s);  // the old table may still be read
            if (e != cudaSuccess) return cuda_fail(e, "batch items resize");
            cudaFree(b->d_items);
            b->d_items = nullptr;
        }
        cudaError_t e = cudaMalloc(&b->d_items, std::max<size_t>(items.size(), 1) * sizeof(BatchItem));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc batch items");
        b->items_cap = items.size();
    }
    if (!items.empty()) {
        cudaError_t e =
            cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "copy batch items");
        e = cudaStreamSynchronize(s);  // `items` is a host temporary
        if (e != cudaSuccess) return cuda_fail(e, "copy batch items");
    }
    b->a.items = b->d_items;
    b->a.n_items = (int64_t)items.size();
    b->a.chunk = chunk;
    return BEZ_OK;
}

bez_status run_setup(bez_batch b, cudaStream_t s)
{
    const LaunchHooks h{no_count, no_event, no_event, nullptr, b->ctx->sm_count};
    int k = 0;
    // the setup kernel alone: an evaluator launch over zero items does no work
    BatchArgs a = b->a;
    a.n_items = 0;
    for (int k = 0; k < 16; ++k) a.class_start[k] = 0;
    cudaError_t e = launch_batch(a, b->shape.threads, b->ctx->sm_count, true, s, nullptr, h, &k);
    if (e != cudaSuccess) return cuda_fail(e, "batch setup");
    b->spans_ready = true;
    return BEZ_OK;
}

bez_status apply_shape(bez_batch b, const Shape& sh, cudaStream_t s)
{
    if (b->a.chunk != sh.chunk || !b->a.items) {
        bez_status st = build_items(b, sh.chunk, s);
        if (st != BEZ_OK) return st;
    }
    const bool repr_changed = b->a.repr != sh.repr;
    b->a.schedule = sh.schedule;
    b->a.grab = 4;
    b->a.partition = 0;
    b->a.repr = sh.repr;
    b->a.op_pool = sh.repr == 1 ? b->d_ops_c : b->d_ops;
    b->shape = sh;
    if (repr_changed || !b->spans_ready) return run_setup(b, s);
    return BEZ_OK;
}

// time one shape (setup included when it runs on every launch): median of 3
// after a warm-up
bez_status time_shape(bez_batch b, const Shape& sh, cudaStream_t s, float* ms_out)
{
    bez_status st = apply_shape(b, sh, s);
    if (st != BEZ_OK) return st;
    const LaunchHooks h{no_count, no_event, no_event, nullptr, b->ctx->sm_count};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float t[3];
    int k = 0;
    cudaError_t e = launch_batch(b->a, sh.threads, b->ctx->sm_count, b->setup_each, s, streams_of(b), h, &k);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
        cudaEventRecord(e0, s);
        e = launch_batch(b->a, sh.threads, b->ctx->sm_count, b->setup_each, s, streams_of(b), h, &k);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&t[r], e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "autotune launch");
    std::sort(t, t + 3);
    *ms_out = t[1];
    return BEZ_OK;
}

// Time `a` (a copy of the plan's arguments): median of 3 after a warm-up.
bez_status time_args(bez_batch b, const BatchArgs& a, bool with_setup, cudaStream_t s, float* ms_out)
{
    const LaunchHooks h{no_count, no_event, no_event, nullptr, b->ctx->sm_count};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float t[3];
    int k = 0;
    cudaError_t e = launch_batch(a, b->shape.threads, b->ctx->sm_count, with_setup, s, streams_of(b), h, &k);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
        cudaEventRecord(e0, s);
        e = launch_batch(a, b->shape.threads, b->ctx->sm_count, with_setup, s, streams_of(b), h, &k);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&t[r], e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "autotune launch");
    std::sort(t, t + 3);
    *ms_out = t[1];
    return BEZ_OK;
}

// Partition the GPU between the class kernels (atomic schedule, shape
// already applied): time every class alone on the whole GPU, give class k
// ceil(G_k t_k / sum t) blocks (G_k its persistent grid), so that all
// classes run side by side and end together.  Sets b->a.partition and the
// grids; `ms_out` is the partitioned launch's time.
bez_status tune_partition(bez_batch b, cudaStream_t s, float* ms_out)
{
    BatchArgs& a = b->a;
    float tc[kBatchClasses] = {};
    float total = 0.f;
    for (int cls = 0; cls < kBatchClasses; ++cls) {
        const int64_t first = a.class_start[cls], last = a.class_start[cls + 1];
        if (last <= first) continue;
        BatchArgs one = a;
        one.partition = 0;
        for (int k = 0; k < 16; ++k) one.class_start[k] = k <= cls ? first : last;
        bez_status st = time_args(b, one, false, s, &tc[cls]);
        if (st != BEZ_OK) return st;
        total += tc[cls];
    }
    for (int k = 0; k < 16; ++k) a.class_grid[k] = 0;
    for (int cls = 0; cls < kBatchClasses && total > 0.f; ++cls) {
        if (tc[cls] <= 0.f) continue;
        const int full = batch_full_grid(a, b->shape.threads, b->ctx->sm_count, cls);
        const int g = (int)std::ceil((double)full * tc[cls] / total);
        a.class_grid[cls] = std::max(1, std::min(full, g));
    }
    a.partition = 1;
    return time_args(b, a, b->setup_each, s, ms_out);
}

bez_status autotune(bez_batch b, cudaStream_t s)
{
    const char* path = getenv("BEZ_AUTOTUNE_CACHE");
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        if (path) load_cache_file(path);
        auto it = g_tune_cache.find(b->key);
        if (it != g_tune_cache.end()) {
            const Shape sh = it->second;
            bez_status st = apply_shape(b, sh, s);
            if (st != BEZ_OK || !sh.partition) return st;
            float ms = 0.f;
            st = tune_partition(b, s, &ms);
            b->shape.partition = 1;
            return st;
        }
    }
    Shape best;
    float best_ms = 1e30f;
    for (int repr : {1, 0})
    for (int chunk : {256, 512, 1024, 2048})
        for (int sched : {0, 1})
            for (int threads : {128, 256}) {
                Shape sh{chunk, sched, threads, repr};
                float ms = 0.f;
                bez_status st = time_shape(b, sh, s, &ms);
                if (st != BEZ_OK) return st;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = sh;
                }
            }
    bez_status st = apply_shape(b, best, s);
    if (st != BEZ_OK) return st;
    if (best.schedule == 1) {
        // the best shape with the GPU partitioned between the classes
        float ms = 0.f;
        st = tune_partition(b, s, &ms);
        if (st != BEZ_OK) return st;
        if (ms < best_ms) {
            best.partition = 1;
            b->shape.partition = 1;
        } else {
            b->a.partition = 0;
        }
    }
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune_cache[b->key] = best;
        if (path) save_cache_file(path);
    }
    return BEZ_OK;
}

void free_batch(bez_batch b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->have_streams) {
        for (int i = 0; i < kBatchSideStreams; ++i) {
            cudaStreamDestroy(b->streams.side[i]);
            cudaEventDestroy(b->streams.join[i]);
        }
        cudaEventDestroy(b->streams.fork);
    }
    cudaFree(b->d_desc);
    cudaFree(b->d_ops);
    cudaFree(b->d_ops_c);
    cudaFree(b->d_span_rec);
    cudaFree(b->d_items);
    cudaFree(b->d_spans);
    cudaFree(b->d_counter);
    delete b;
}

}  // namespace

extern "C" {

bez_status bez_batch_create(bez_ctx c, const bez_curve_desc* desc, int64_t n_curves, int dim, const float* ctrl_pool,
                            int64_t ctrl_len, const float* weight_pool, int64_t weight_len, float* out_pool,
                            int64_t out_len, const bez_batch_opts* bo, void* stream, bez_batch* out)
{
    if (!out) return fail(BEZ_ERR_INVALID_ARG, "null output handle");
    *out = nullptr;
    if (!c) return fail(BEZ_ERR_INVALID_ARG, "null context");
    if (n_curves < 0 || ctrl_len < 0 || weight_len < 0 || out_len < 0) return fail(BEZ_ERR_INVALID_ARG, "negative size");
    if (n_curves > 0x7fffffff) return fail(BEZ_ERR_INVALID_ARG, "more than 2^31-1 curves");
    if (dim < 1 || dim > 4) return fail(BEZ_ERR_INVALID_ARG, "dim %d not in 1..4", dim);
    if (n_curves > 0 && !desc) return fail(BEZ_ERR_INVALID_ARG, "null descriptors");
    std::lock_guard<std::mutex> g(c->mu);
    BEZ_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((ctrl_len > 0 && classify(ctrl_pool) != MEM_DEVICE) || (out_len > 0 && classify(out_pool) != MEM_DEVICE) ||
        (weight_len > 0 && classify(weight_pool) != MEM_DEVICE))
        return fail(BEZ_ERR_INVALID_ARG, "batch pools must be device arrays");
    bez_batch b = new bez_batch_s();
    b->ctx = c;
    b->hdesc.resize((size_t)n_curves);
    if (n_curves > 0) {
        const cudaMemcpyKind kind = classify(desc) == MEM_DEVICE ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        cudaError_t e = cudaMemcpy(b->hdesc.data(), desc, (size_t)n_curves * sizeof(bez_curve_desc), kind);
        if (e != cudaSuccess) {
            delete b;
            return cuda_fail(e, "copy descriptors");
        }
    }
    // validate every descriptor against the pools
    std::vector<int64_t> span_off((size_t)n_curves, 0), op_off((size_t)n_curves, 0);
    std::map<std::pair<int, int>, int64_t> op_index;   // (n_ctrl, degree) -> offset into span_ops
    std::map<std::vector<long long>, int64_t> mat_index;  // distinct matrices -> offset into ops
    std::vector<int64_t> span_ops;                       // per span: offset of its matrix in ops
    std::vector<double> ops;
    std::vector<std::pair<int64_t, int>> mats;           // (offset, degree) of every distinct matrix
    int64_t spans = 0, total_samples = 0, n_type[3] = {0, 0, 0}, deg_sum = 0;
    for (int64_t i = 0; i < n_curves; ++i) {
        const bez_curve_desc& d = b->hdesc[(size_t)i];
        const char* why = nullptr;
        if (d.type < BEZ_CURVE_BEZIER || d.type > BEZ_CURVE_NURBS) why = "unknown curve type";
        else if (d.degree < 1 || d.degree > 7) why = "degree outside 1..7";
        else if (d.type == BEZ_CURVE_BEZIER && d.n_ctrl != d.degree + 1) why = "a Bezier curve has degree+1 points";
        else if (d.n_ctrl < d.degree + 1) why = "fewer than degree+1 control points";
        else if (d.n_samples < 0) why = "negative sample count";
        else if (d.ctrl_off < 0 || d.ctrl_off + (int64_t)d.n_ctrl * dim > ctrl_len) why = "control points outside ctrl_pool";
        else if (d.out_off < 0 || d.out_off + (int64_t)d.n_samples * dim > out_len) why = "samples outside out_pool";
        else if (d.type == BEZ_CURVE_NURBS && (!weight_pool || d.weight_off < 0 || d.weight_off + d.n_ctrl > weight_len))
            why = "weights outside weight_pool";
        if (why) {
            delete b;
            return fail(BEZ_ERR_INVALID_ARG, "curve %lld: %s", (long long)i, why);
        }
        n_type[d.type] += 1;
        deg_sum += d.degree;
        total_samples += d.n_samples;
        const int comps = d.type == BEZ_CURVE_NURBS ? dim + 1 : dim;
        const int n_spans = d.type == BEZ_CURVE_BEZIER ? 1 : d.n_ctrl - d.degree;
        span_off[(size_t)i] = spans;
        spans += (int64_t)n_spans * kSpanStride(d.degree, comps);  // stays a multiple of 4 floats
        if (d.type != BEZ_CURVE_BEZIER) {
            // knot insertion once per distinct (n_ctrl, degree), in FP64
            const auto key = std::make_pair(d.n_ctrl, d.degree);
            auto it = op_index.find(key);
            if (it == op_index.end()) {
                // operators of every span, de-duplicated: on clamped uniform
                // knots all interior spans of one degree share one matrix
                const int p = d.degree, sq = (p + 1) * (p + 1);
                const int64_t off = (int64_t)span_ops.size();
                std::vector<double> M((size_t)sq);
                for (int k = p; k < d.n_ctrl; ++k) {
                    span_operator(nullptr, d.n_ctrl, p, k, M.data());
                    std::vector<long long> mk(1, p);
                    for (double v : M) mk.push_back(std::llround(v * 1099511627776.0));  // 2^40
                    auto mt = mat_index.find(mk);
                    if (mt == mat_index.end()) {
                        // rows padded to an even length (zeros) so the device
                        // reads each row as 16-byte pairs of entries
                        mt = mat_index.emplace(mk, (int64_t)ops.size()).first;
                        mats.emplace_back((int64_t)ops.size(), p);
                        const int stride = kOpRowStride(p);
                        for (int i = 0; i <= p; ++i) {
                            ops.insert(ops.end(), M.begin() + i * (p + 1), M.begin() + (i + 1) * (p + 1));
                            ops.insert(ops.end(), (size_t)(stride - (p + 1)), 0.0);
                        }
                    }
                    span_ops.push_back(mt->second);
                }
                it = op_index.emplace(key, off).first;
            }
            op_off[(size_t)i] = it->second;
        }
    }
    // plan-owned device buffers
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    };
    alloc((void**)&b->d_desc, (size_t)n_curves * sizeof(bez_curve_desc));
    // Centred representation: the Bezier -> power-basis-about-1/2 map is a
    // fixed matrix T_p per degree, so each span operator M becomes T_p M (FP64
    // here) and a Bezier curve's span uses T_p itself; the device then forms
    // either representation with the same compensated dot products.  Both
    // pools share one layout: the distinct M, then T_1 .. T_7.
    std::vector<double> ops_c(ops.size(), 0.0);
    for (const auto& mp : mats) {
        const int p = mp.second, st = kOpRowStride(p);
        double T[8][8];
        centred_matrix(p, T);
        for (int i = 0; i <= p; ++i)
            for (int j = 0; j <= p; ++j) {
                double acc = 0.0;
                for (int k = 0; k <= p; ++k) acc += T[i][k] * ops[(size_t)(mp.first + (int64_t)k * st + j)];
                ops_c[(size_t)(mp.first + (int64_t)i * st + j)] = acc;
            }
    }
    for (int p = 1; p <= 7; ++p) {
        const int st = kOpRowStride(p);
        b->a.tpow_off[p] = (int64_t)ops.size();
        double T[8][8];
        centred_matrix(p, T);
        for (int i = 0; i <= p; ++i)
            for (int j = 0; j < st; ++j) {
                ops.push_back(j == i ? 1.0 : 0.0);  // unused in the Bezier-point pool
                ops_c.push_back(j <= p ? T[i][j] : 0.0);
            }
    }
    b->a.tpow_off[0] = 0;
    // operators as unevaluated float pairs hi + lo: hi = fl32(M), lo = fl32(M - hi)
    auto split = [](const std::vector<double>& v) {
        std::vector<float2> r(v.size());
        for (size_t k = 0; k < v.size(); ++k) {
            const float hi = (float)v[k];
            r[k] = make_float2(hi, (float)(v[k] - (double)hi));
        }
        return r;
    };
    const std::vector<float2> ops2 = split(ops), ops2c = split(ops_c);
    alloc((void**)&b->d_ops, ops2.size() * sizeof(float2));
    alloc((void**)&b->d_ops_c, ops2c.size() * sizeof(float2));
    alloc((void**)&b->d_spans, (size_t)spans * sizeof(float));
    alloc(&b->d_counter, kBatchClasses * sizeof(unsigned long long));
    // every span with its offsets resolved, grouped by item class (so that a
    // class's spans can be extracted on its own stream just before its
    // evaluator) and within a class by (degree, type) (so that the warps of
    // the setup kernel run one degree's code at a time)
    std::vector<int64_t> order((size_t)n_curves);
    for (int64_t i = 0; i < n_curves; ++i) order[(size_t)i] = i;
    auto span_key = [&](int64_t i) {
        const bez_curve_desc& d = b->hdesc[(size_t)i];
        return ((int64_t)batch_item_class(d, dim) * 64 + d.degree) * 4 + d.type;
    };
    std::stable_sort(order.begin(), order.end(),
                     [&](int64_t x, int64_t y) { return span_key(x) < span_key(y); });
    std::vector<SpanRec> span_rec;
    int64_t span_class_start[16] = {};
    {
        int cls_next = 0;
        for (int64_t i : order) {
            const bez_curve_desc& d = b->hdesc[(size_t)i];
            const int cls = batch_item_class(d, dim);
            while (cls_next <= cls) span_class_start[cls_next++] = (int64_t)span_rec.size();
            {
                const bool spline = d.type != BEZ_CURVE_BEZIER, rat = d.type == BEZ_CURVE_NURBS;
                const int comps = rat ? dim + 1 : dim;
                const int n_spans = spline ? d.n_ctrl - d.degree : 1;
                for (int s = 0; s < n_spans; ++s) {
                    SpanRec r{};
                    r.ctrl = d.ctrl_off + (int64_t)s * dim;
                    r.weight = rat ? d.weight_off + s : -1;
                    r.dst = span_off[(size_t)i] + (int64_t)s * kSpanStride(d.degree, comps);
                    r.op = spline ? span_ops[(size_t)(op_off[(size_t)i] + s)] : -1;
                    r.degree = d.degree;
                    r.type = d.type;
                    span_rec.push_back(r);
                }
            }
        }
        while (cls_next < 16) span_class_start[cls_next++] = (int64_t)span_rec.size();
    }
    alloc((void**)&b->d_span_rec, span_rec.size() * sizeof(SpanRec));
    if (e == cudaSuccess && !span_rec.empty())
        e = cudaMemcpy(b->d_span_rec, span_rec.data(), span_rec.size() * sizeof(SpanRec), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && n_curves > 0)
        e = cudaMemcpy(b->d_desc, b->hdesc.data(), (size_t)n_curves * sizeof(bez_curve_desc), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !ops.empty())
        e = cudaMemcpy(b->d_ops, ops2.data(), ops2.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !ops2c.empty())
        e = cudaMemcpy(b->d_ops_c, ops2c.data(), ops2c.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "batch buffers");
    }
    b->hspan_off = std::move(span_off);
    // side streams for the class evaluators (joined back on every launch)
    {
        BatchStreams& st = b->streams;
        const bool have_fork = cudaEventCreateWithFlags(&st.fork, cudaEventDisableTiming) == cudaSuccess;
        bool ok = have_fork;
        int ns = 0, ne = 0;
        for (int i = 0; ok && i < kBatchSideStreams; ++i) {
            ok = cudaStreamCreateWithFlags(&st.side[i], cudaStreamNonBlocking) == cudaSuccess;
            if (ok) ++ns;
            if (ok) ok = cudaEventCreateWithFlags(&st.join[i], cudaEventDisableTiming) == cudaSuccess;
            if (ok) ++ne;
        }
        if (!ok) {
            for (int i = 0; i < ns; ++i) cudaStreamDestroy(st.side[i]);
            for (int i = 0; i < ne; ++i) cudaEventDestroy(st.join[i]);
            if (have_fork) cudaEventDestroy(st.fork);
            cudaGetLastError();
            free_batch(b);
            return fail(BEZ_ERR_CUDA, "batch side streams");
        }
        b->have_streams = true;
    }
    BatchArgs& a = b->a;
    a.desc = b->d_desc;
    a.n_curves = n_curves;
    a.dim = dim;
    a.ctrl_pool = ctrl_pool;
    a.weight_pool = weight_pool;
    a.out_pool = out_pool;
    a.span_pool = b->d_spans;
    a.op_pool = b->d_ops;
    a.span_rec = b->d_span_rec;
    a.n_span_rec = (int64_t)span_rec.size();
    for (int k = 0; k < 16; ++k) a.span_class_start[k] = span_class_start[k];
    a.repr = -1;  // set by apply_shape, which then runs the setup
    a.counter = b->d_counter;
    b->setup_each = bo ? bo->setup_each_launch != 0 : true;
    b->use_graph = bo ? bo->use_graph != 0 : false;
    char key[160];
    snprintf(key, sizeof(key), "batch-v3:setup%d:n%d:dim%d:mix%lld/%lld/%lld:deg%d:s%d", b->setup_each ? 1 : 0,
             log2_bucket((double)n_curves), dim,
             (long long)(n_curves ? 100 * n_type[0] / n_curves : 0), (long long)(n_curves ? 100 * n_type[1] / n_curves : 0),
             (long long)(n_curves ? 100 * n_type[2] / n_curves : 0), n_curves ? (int)std::lround((double)deg_sum / n_curves) : 0,
             log2_bucket(n_curves ? (double)total_samples / n_curves : 0.0));
    b->key = key;
    // launch shape: explicit, tuned or default
    Shape sh;
    if (bo && bo->chunk > 0) sh.chunk = bo->chunk;
    if (bo && (bo->schedule == 0 || bo->schedule == 1)) sh.schedule = bo->schedule;
    const bool want_partition = bo && bo->schedule == 2;  // atomic queue, GPU partitioned between the classes
    if (want_partition) sh.schedule = 1;
    if (bo && (bo->threads == 128 || bo->threads == 256)) sh.threads = bo->threads;
    if (bo && (bo->repr == 0 || bo->repr == 1)) sh.repr = bo->repr;
    if (bo && bo->chunk > 0 && bo->chunk % 256 != 0) {
        free_batch(b);
        return fail(BEZ_ERR_INVALID_ARG, "chunk must be a multiple of 256");
    }
    if (bo && bo->threads != 0 && bo->threads != 128 && bo->threads != 256) {
        free_batch(b);
        return fail(BEZ_ERR_INVALID_ARG, "threads must be 128 or 256");
    }
    bez_status st = BEZ_OK;
    if (st == BEZ_OK) st = (bo && bo->autotune) ? autotune(b, s) : apply_shape(b, sh, s);
    if (st == BEZ_OK && want_partition && !(bo && bo->autotune)) {
        float ms = 0.f;
        st = tune_partition(b, s, &ms);
        b->shape.partition = 1;
    }
    if (st == BEZ_OK && b->use_graph) {
        cudaStream_t cs = nullptr;
        cudaGraph_t graph = nullptr;
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const LaunchHooks h0{no_count, no_event, no_event, nullptr, c->sm_count};
            int k = 0;
            cudaError_t le = launch_batch(a, b->shape.threads, c->sm_count, b->setup_each, cs, streams_of(b), h0, &k);
            e = cudaStreamEndCapture(cs, &graph);
            if (le != cudaSuccess) e = le;
            b->kernels_per_launch = k;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
        if (e != cudaSuccess) st = cuda_fail(e, "batch graph capture");
    }
    if (st != BEZ_OK) {
        cudaStreamSynchronize(s);
        free_batch(b);
        return st;
    }
    *out = b;
    return BEZ_OK;
}

bez_status bez_batch_launch(bez_batch b, void* stream)
{
    if (!b) return fail(BEZ_ERR_INVALID_ARG, "null batch");
    bez_ctx c = b->ctx;
    std::lock_guard<std::mutex> g(c->mu);
    BEZ_CUDA(cudaSetDevice(c->device), "cudaSetDevice");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LaunchHooks h = hooks_of(c);
    if (b->exec) {
        for (int i = 0; i < b->kernels_per_launch; ++i) h.count(h.self);
        h.begin(h.self, s);
        cudaError_t e = cudaGraphLaunch(b->exec, s);
        h.end(h.self, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
        return BEZ_OK;
    }
    int k = 0;
    cudaError_t e = launch_batch(b->a, b->shape.threads, c->sm_count, b->setup_each, s, streams_of(b), h, &k);
    if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    return BEZ_OK;
}

bez_status bez_batch_config(bez_batch b, int32_t* chunk, int32_t* schedule, int32_t* threads, int32_t* repr)
{
    if (!b) return fail(BEZ_ERR_INVALID_ARG, "null batch");
    if (repr) *repr = b->shape.repr;
    if (chunk) *chunk = b->shape.chunk;
    if (schedule) *schedule = b->shape.schedule == 1 && b->shape.partition ? 2 : b->shape.schedule;
    if (threads) *threads = b->shape.threads;
    return BEZ_OK;
}

bez_status bez_batch_destroy(bez_batch b)
{
    if (!b) return BEZ_OK;
    cudaSetDevice(b->ctx->device);
    cudaDeviceSynchronize();
    free_batch(b);
    return BEZ_OK;
}

bez_status bez_eval_batch(bez_ctx c, const bez_curve_desc* desc, int64_t n_curves, int dim, const float* ctrl_pool,
                          int64_t ctrl_len, const float* weight_pool, int64_t weight_len, float* out_pool,
                          int64_t out_len, void* stream)
{
    bez_batch_opts bo{0, 1, 0, 0, -1, 0, -1};
    bez_batch b = nullptr;
    bez_status st = bez_batch_create(c, desc, n_curves, dim, ctrl_pool, ctrl_len, weight_pool, weight_len, out_pool,
                                     out_len, &bo, stream, &b);
    if (st != BEZ_OK) return st;
    st = bez_batch_launch(b, stream);
    cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    bez_batch_destroy(b);
    return st;
}

}  // extern "C"
