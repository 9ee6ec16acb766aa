// tensor_common.cuh -- pieces shared by the CUDA-core and texture
// tensor-product kernels: the kernel-side argument block and the Bernstein
// tables of the uniform grid values.
#pragma once

#include "curve_eval.cuh"

namespace bez {

constexpr int kTensorThreads = 256;
constexpr int kTensorMaxDeg = 7;
constexpr int kTensorMaxGrid = 256;

struct TensorArgs {  // kernel-side copy of TensorLaunch
    const void* ctrl;
    int32_t dtype;
    int64_t n;
    int32_t du, dv, dw;  // dw < 0: surface
    int32_t dim;
    int32_t nu, nv, nw;
    float* out;
};

// Bernstein table B[a][i] for n grid values and degree d, via de Casteljau
// on unit vectors (each entry is a product of lerp weights, exact at ends).
__device__ __forceinline__ void bernstein_table(float* B, int n, int d, int tid, int nthreads)
{
    for (int a = tid; a < n; a += nthreads) {
        const float t = n > 1 ? __fdiv_rn((float)a, (float)(n - 1)) : 0.f;
        const float s = 1.0f - t;
        // B_i^d(t) = C(d,i) s^(d-i) t^i, built from powers
        float tp[kTensorMaxDeg + 1], sp[kTensorMaxDeg + 1];
        tp[0] = sp[0] = 1.f;
        for (int i = 1; i <= d; ++i) {
            tp[i] = tp[i - 1] * t;
            sp[i] = sp[i - 1] * s;
        }
        float bin = 1.f;
        for (int i = 0; i <= d; ++i) {
            B[a * (d + 1) + i] = bin * sp[d - i] * tp[i];
            bin = bin * (float)(d - i) / (float)(i + 1);
        }
    }
}

// warp-per-patch kernels: warps per block and the largest u grid they hold
constexpr int kSurfWarps = 8;
constexpr int kSurfMaxRows = 64;

}  // namespace bez
