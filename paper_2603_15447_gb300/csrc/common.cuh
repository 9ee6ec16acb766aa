// common.cuh -- device helpers shared by the libbez kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace bez {

constexpr int kMaxDegree = 15;   // register evaluators: degree 1..15
constexpr unsigned kFull = 0xffffffffu;

// parameter-stream kinds as seen by kernels (the C enum's SHARED / PER_CURVE
// both become TM_ARRAY with a per-curve stride of 0 or n_t)
// TM_HASH16: the same draw as TM_HASH when every sample index is < 2^16, with
// the per-curve key pre-mixed (lowbias32_premixed).
enum { TM_ARRAY = 0, TM_UNIFORM = 1, TM_HASH = 2, TM_HASH16 = 3 };
enum { OM_POINTS = 0, OM_LENGTH = 1 };
enum { VAR_HORNER = 1, VAR_HORNER_CENTRED = 2, VAR_BERNSTEIN = 3, VAR_DECASTELJAU = 4, VAR_SEILER = 5 };

__host__ __device__ constexpr int binom_c(int n, int k)
{
    return (k < 0 || k > n) ? 0 : (k == 0 || k == n) ? 1 : binom_c(n - 1, k - 1) + binom_c(n - 1, k);
}

// lowbias32 (C. Wellons, 2018): xorshift-multiply integer mixer.
__host__ __device__ __forceinline__ uint32_t lowbias32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

constexpr uint32_t kLowbiasMul1 = 0x7feb352du;

// lowbias32 from its first product on: y = (x ^ (x >> 16)) * 0x7feb352d
__device__ __forceinline__ uint32_t lowbias32_tail(uint32_t y)
{
    y ^= y >> 15;
    y *= 0x846ca68bu;
    y ^= y >> 16;
    return y;
}

// lowbias32(k ^ j) for j < 2^16, given km = k ^ (k >> 16): the first
// xorshift distributes over the xor and j >> 16 == 0, so
// (k ^ j) ^ ((k ^ j) >> 16) == km ^ j.  Same value, two instructions fewer.
__device__ __forceinline__ uint32_t lowbias32_premixed(uint32_t km, uint32_t j)
{
    return lowbias32_tail((km ^ j) * kLowbiasMul1);
}

// 1 + (23 high bits of h) 2^-23, in [1,2): (0x7f : h) >> 9 == 0x3f800000 | (h >> 9),
// so one funnel shift builds the float 1.m
__device__ __forceinline__ float hash_one_plus(uint32_t h)
{
    return __uint_as_float(__funnelshift_r(h, 0x7fu, 9));
}

// 23 high bits of h as a uniform in [0,1): 1.m - 1 is exact in FP32.
__device__ __forceinline__ float hash_unit(uint32_t h)
{
    return hash_one_plus(h) - 1.0f;
}

// a + t (b - a) written as (a - t a) + t b: exact at t = 0 and t = 1, and
// lerp(a, a, t) == a for every t in [0, 1].
__device__ __forceinline__ float lerp(float a, float b, float t)
{
    return fmaf(t, b, fmaf(-t, a, a));
}

// clamp to [0,1] keeping NaN (fminf/fmaxf would drop it)
__device__ __forceinline__ float clamp01(float t)
{
    return t < 0.f ? 0.f : (t > 1.f ? 1.f : t);
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float load_elem(const void* p, int dtype, int64_t i)
{
    if (dtype == 0) return __ldg(static_cast<const float*>(p) + i);
    if (dtype == 1) return __half2float(static_cast<const __half*>(p)[i]);
    return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Warp totals of 16 values by recursive halving (a reduce-scatter): at each
// level a lane keeps one half of its values, sends the other half to its
// partner and adds what the partner sent for the kept half.  Returns, in
// lanes 2i and 2i + 1, the warp total of v[i]; 16 shuffles instead of the
// 80 of sixteen butterflies.  v is overwritten.
__device__ __forceinline__ float warp_sum16_scatter(float (&v)[16], int lane)
{
#pragma unroll
    for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = upper ? v[i] : v[i + h];
            const float keep = upper ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(kFull, send, o);
        }
    }
    return v[0] + __shfl_xor_sync(kFull, v[0], 1);
}

}  // namespace bez
