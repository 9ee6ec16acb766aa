// context.h -- the libbez context object and host helpers shared by the
// runtime translation units (api.cu, batch_plan.cu).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/bez.h"
#include "internal.h"

struct StageBuf {
    void* p = nullptr;
    size_t cap = 0;
};

struct bez_ctx_s {
    int device = 0;
    int sm_count = 0;
    bool timing = false;
    int64_t launches = 0;
    int64_t timed_launches = 0;
    double timed_ms = 0.0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    std::vector<cudaEvent_t> spare;
    cudaEvent_t cur_begin = nullptr;
    StageBuf stage[9];  // 0 ctrl, 1 t, 2 out, 3 weights, 4 knots / grad_out / targets, 6-8 extra outputs (host
                        // staging); 5 spline spans (scratch)
    bez::TexState tex;
    // pipelined host calls: chunk copies in and out on their own streams
    cudaStream_t pipe_in = nullptr, pipe_out = nullptr;
    cudaStream_t pipe_alt = nullptr;  // odd chunks evaluate here, so a chunk's tail overlaps the next chunk
    cudaEvent_t pipe_ev[2 * 8 + 2] = {};  // start, per chunk in / done (8 chunks at most), end
    cudaEvent_t tex_done = nullptr;  // last use of the texture atlases
    bool tex_used = false;
    std::mutex mu;
};


#define BEZ_CUDA(call, what)                                       \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return bez::cuda_fail(e_, (what));  \
    } while (0)

namespace bez {
bez_status fail(bez_status st, const char* fmt, ...);
bez_status cuda_fail(cudaError_t e, const char* what);
LaunchHooks hooks_of(bez_ctx c);
enum MemKind { MEM_NULL, MEM_DEVICE, MEM_HOST };
MemKind classify(const void* p);
}  // namespace bez
