// internal.h -- declarations shared between the libbez host runtime and the
// kernel translation units.  Not part of the public ABI (see include/bez.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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
};

// Result of a launcher: how many kernels it launched and the CUDA status.
struct LaunchResult {
    int launches;
    cudaError_t err;
};

// Hooks the runtime passes to launchers so that the main kernel of a call is
// bracketed by timing events and counted.
struct LaunchHooks {
    void (*begin)(void* self, cudaStream_t s);
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

// Occupancy-sized persistent grid: a multiple of the SM count.
int persistent_grid(const void* kernel, int block, size_t smem, int sm_count, int64_t work_blocks);

}  // namespace bez
