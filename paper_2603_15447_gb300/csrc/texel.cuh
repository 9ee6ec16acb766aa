// texel.cuh -- one RGBA texel of an atlas written in its storage format
// (float4, half4, or unorm16 / unorm8 codes of a value already mapped to
// [0, 1] by its tile's rescale).
#pragma once

#include "common.cuh"

namespace bez {

// storage formats of an atlas
enum { TEXEL_F32 = 0, TEXEL_F16 = 1, TEXEL_UNORM16 = 2, TEXEL_UNORM8 = 3 };

// unorm code of a value in [0, 1] with `levels` = 2^bits - 1, round to nearest
__device__ __forceinline__ unsigned unorm_code(float v, float levels)
{
    const float x = fminf(fmaxf(v, 0.f), 1.f) * levels;
    return (unsigned)__float2uint_rn(x);
}

__device__ __forceinline__ void put(cudaSurfaceObject_t s, int fmt, int x, int y, int z, bool is3d, float4 v)
{
    if (fmt == TEXEL_F32) {
        if (is3d) surf3Dwrite(v, s, x * 16, y, z);
        else surf2Dwrite(v, s, x * 16, y);
    } else if (fmt == TEXEL_F16) {
        const __half2 lo = __floats2half2_rn(v.x, v.y), hi = __floats2half2_rn(v.z, v.w);
        const uint2 bits = make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
        if (is3d) surf3Dwrite(bits, s, x * 8, y, z);
        else surf2Dwrite(bits, s, x * 8, y);
    } else if (fmt == TEXEL_UNORM16) {
        const ushort4 u = make_ushort4(unorm_code(v.x, 65535.f), unorm_code(v.y, 65535.f), unorm_code(v.z, 65535.f),
                                       unorm_code(v.w, 65535.f));
        if (is3d) surf3Dwrite(u, s, x * 8, y, z);
        else surf2Dwrite(u, s, x * 8, y);
    } else {
        const uchar4 u = make_uchar4(unorm_code(v.x, 255.f), unorm_code(v.y, 255.f), unorm_code(v.z, 255.f),
                                     unorm_code(v.w, 255.f));
        if (is3d) surf3Dwrite(u, s, x * 4, y, z);
        else surf2Dwrite(u, s, x * 4, y);
    }
}

__device__ __forceinline__ float4 min4(float4 a, float4 b)
{
    return make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z), fminf(a.w, b.w));
}
__device__ __forceinline__ float4 max4(float4 a, float4 b)
{
    return make_float4(fmaxf(a.x, b.x), fmaxf(a.y, b.y), fmaxf(a.z, b.z), fmaxf(a.w, b.w));
}

}  // namespace bez
