// peaks.cu -- microbenchmarks that give the roofline denominators of the
// evaluators: FP32 FMA issue rate, linear-filtered texture fetch rates
// (2D bilinear / 3D trilinear, float4 / half4 texels, L1-resident textures),
// and device-memory store / copy bandwidth.  Each kernel is timed with CUDA
// events on the caller's stream after a warm-up launch.
#include <functional>

#include "curve_eval.cuh"

namespace bez {

constexpr int kPeakThreads = 256;

// 8 independent FMA chains per thread; the result is stored only if it is
// impossible in practice, so the work cannot be removed.
__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(float seed, int iters, float* sink)
{
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed + threadIdx.x * 1e-7f + k;
    const float m = 0.9999999f, c = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 12345.678f) sink[0] = s;
}

// fetches at coordinates that move every iteration (no reuse of a result)
template <bool IS3D>
__global__ void __launch_bounds__(kPeakThreads) k_peak_tex(cudaTextureObject_t tex, int iters, float* sink)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    float x = 1.5f + (tid & 31) * 0.37f, y = 1.5f + ((tid >> 5) & 7) * 0.61f, z = 0.75f;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = 0; i < iters; ++i) {
        const float4 v = IS3D ? tex3D<float4>(tex, x, y, z) : tex2D<float4>(tex, x, y);
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
        x += 0.0137f;
        y += 0.0071f;
        if (x > 60.f) x -= 58.f;
        if (y > 60.f) y -= 58.f;
    }
    if (acc.x + acc.y + acc.z + acc.w == 12345.678f) sink[0] = acc.x;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_store(float4* dst, int64_t n4)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride)
        dst[i] = make_float4(1.f, 2.f, 3.f, (float)i);
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_copy(const float4* __restrict__ src, float4* dst, int64_t n4)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) dst[i] = src[i];
}

static cudaError_t time_launch(cudaStream_t s, float* ms, const std::function<void()>& launch)
{
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    cudaEventCreate(&e1);
    launch();  // warm-up
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

cudaError_t measure_peak(int kind, int sm_count, cudaStream_t s, double* value)
{
    float* sink = nullptr;
    cudaError_t e = cudaMalloc(&sink, 16);
    if (e != cudaSuccess) return e;
    float ms = 0.f;
    if (kind == 0) {  // FP32 FMA lane operations per second
        const int blocks = sm_count * 8, iters = 1 << 14;
        e = time_launch(s, &ms, [&] { k_peak_fma<<<blocks, kPeakThreads, 0, s>>>(1.f, iters, sink); });
        *value = (double)blocks * kPeakThreads * iters * 8 / (ms * 1e-3);
    } else if (kind >= 1 && kind <= 4) {  // texture fetches per second
        const bool is3d = kind >= 3, half = (kind % 2) == 0;
        Atlas at;
        e = atlas_ensure(at, 64, 64, is3d ? 2 : 0, half ? 1 : 0);
        if (e == cudaSuccess) {
            const int blocks = sm_count * 8, iters = 1 << 12;
            if (is3d)
                e = time_launch(s, &ms, [&] { k_peak_tex<true><<<blocks, kPeakThreads, 0, s>>>(at.tex, iters, sink); });
            else
                e = time_launch(s, &ms, [&] { k_peak_tex<false><<<blocks, kPeakThreads, 0, s>>>(at.tex, iters, sink); });
            *value = (double)blocks * kPeakThreads * iters / (ms * 1e-3);
        }
        atlas_free(at);
    } else {  // device memory GB/s: 5: store, 6: copy (read + write bytes)
        const int64_t bytes = int64_t(2) << 30;
        float4 *a = nullptr, *b = nullptr;
        e = cudaMalloc(&a, bytes);
        if (e == cudaSuccess && kind == 6) e = cudaMalloc(&b, bytes);
        if (e == cudaSuccess) {
            const int64_t n4 = bytes / 16;
            const int blocks = sm_count * 8;
            if (kind == 5) e = time_launch(s, &ms, [&] { k_peak_store<<<blocks, kPeakThreads, 0, s>>>(a, n4); });
            else e = time_launch(s, &ms, [&] { k_peak_copy<<<blocks, kPeakThreads, 0, s>>>(a, b, n4); });
            *value = (double)bytes * (kind == 6 ? 2 : 1) / (ms * 1e-3) / 1e9;
        }
        cudaFree(a);
        cudaFree(b);
    }
    cudaFree(sink);
    return e;
}

}  // namespace bez
