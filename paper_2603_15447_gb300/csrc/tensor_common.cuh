// tensor_common.cuh -- pieces shared by the CUDA-core and texture
// tensor-product kernels: the kernel-side argument block, the Bernstein
// tables of the uniform grid values, and the tricubic scalar volume kernel
// whose u stage runs on either.
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
    int32_t vparts;  // tricubic volume kernel: warps per volume, each a range of u rows (0 = 1)
};

// Warps per volume for the tricubic volume kernel: enough (volume, row
// range) units to fill the SMs about twice over, at most 4 and at most nu.
inline int volume_parts(int64_t n, int nu, int sm_count)
{
    const int64_t target = (int64_t)sm_count * 2 * 32;  // two rounds of 32 resident warps per SM
    int parts = 1;
    while (parts < 4 && parts < nu && n * parts < target) parts *= 2;
    return parts;
}

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

// Texture tiles of the texture surface / volume kernels.
struct SurfTexArgs {
    cudaTextureObject_t tex;
    int tw;                 // tiles per atlas row
    const float4* rescale;  // unorm tiles: (lo, scale) per tile, value = lo + scale x code / levels; else NULL
    int sp;                 // Seiler tiles: texel intervals per tile axis (1: the 2x2 tile read at (u, st);
                            // s >= 2: (s+1) x (s+1) spread tile read at (s u, 4 s st))
};

// Unnormalised coordinates of the Seiler read of tile q at parameter u: the
// paper's 2x2 tile at (u, u (1 - u)), or the spread tile at
// (s u, 4 s u (1 - u)) (the tile's bilinear function sampled on an
// (s+1) x (s+1) grid, see tex.cu).
__device__ __forceinline__ float4 seiler_tile_read(const SurfTexArgs& ta, int64_t q, float u)
{
    const int n1 = ta.sp + 1;
    const float x = (float)((int)(q % ta.tw) * n1) + 0.5f, y = (float)((int)(q / ta.tw) * n1) + 0.5f;
    const float st = fmaf(-u, u, u);
    if (ta.sp == 1) return tex2D<float4>(ta.tex, x + u, y + st);
    const float s = (float)ta.sp;
    return tex2D<float4>(ta.tex, x + s * u, y + (4.f * s) * st);
}

// A filtered unorm read mapped back to values: filtering is affine with
// weights summing to 1, so lo + scale f of the filtered code f.
__device__ __forceinline__ float4 ta_rescale(const SurfTexArgs& ta, int64_t q, float4 f)
{
    const float4 lo = __ldg(ta.rescale + 2 * q), sc = __ldg(ta.rescale + 2 * q + 1);
    return make_float4(fmaf(sc.x, f.x, lo.x), fmaf(sc.y, f.y, lo.y), fmaf(sc.z, f.z, lo.z), fmaf(sc.w, f.w, lo.w));
}

// u stage of the tricubic scalar volume kernel
enum { VOL_U_CORES = 0, VOL_U_TEX_DC = 1, VOL_U_TEX_SEILER = 2 };


// Fast path for tricubic scalar volumes (dim 1, nu <= 32, nw a multiple of
// 4): one warp per volume, no block barrier after the tables.  The warp
// forms Y[a][j][l] = sum_i Bu[a][i] C[i][j][l] in warp-private shared memory
// -- on the FP32 pipes (VOL_U_CORES), or as one filtered read per (a, j) of
// a texture tile whose channel l holds the u cubic C[.][j][l] (de Casteljau
// 2x2x2 tile read at (u, u, u), or the 2x2 Seiler tile read at
// (u, u (1 - u))), the surface construction of Sec. 2.2 / Sec. 4 one axis up --
// then sweeps the u slabs: the slab V[a][.][.] is nv nw consecutive floats,
// and lane l writes its float4s f = l, l + 32, ... (column quad c0 = 4 (f mod
// nw/4) of row b = f div (nw/4)), forming Z[a][b][0..3] = sum_j Bv[b][j]
// Y[a][j][.] for its row and four values sum_l Bw[c][l] Z[a][b][l].  Every
// store instruction writes 512 contiguous bytes.
constexpr int kVolMaxRows = 32;

template <int USTAGE>
__global__ void __launch_bounds__(kSurfWarps * 32) k_volume_tricubic1_warp(const TensorArgs a, const SurfTexArgs ta)
{
    __shared__ float4 s_bu[kVolMaxRows];                      // Bu[a][0..3]
    __shared__ float4 s_bv[kTensorMaxGrid];                   // Bv[b][0..3]
    __shared__ float4 s_bw[kTensorMaxGrid];                   // Bw[c][0..3]
    __shared__ float4 s_y[kSurfWarps][kVolMaxRows * 4];       // Y[a][j][0..3]
    __shared__ float4 s_c4[kSurfWarps][16];                   // C[i][j][0..3]
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    bernstein_table(reinterpret_cast<float*>(s_bu), a.nu, 3, tid, kSurfWarps * 32);
    bernstein_table(reinterpret_cast<float*>(s_bv), a.nv, 3, tid, kSurfWarps * 32);
    bernstein_table(reinterpret_cast<float*>(s_bw), a.nw, 3, tid, kSurfWarps * 32);
    __syncthreads();

    const int nu = a.nu, nv = a.nv, nw = a.nw;
    const int q4 = nw / 4;                // float4 per (a, b) row
    const int slab4 = nv * q4;            // float4 per u slab
    const int64_t pts = (int64_t)nu * nv * nw;
    const int64_t stride = (int64_t)gridDim.x * kSurfWarps;
    const int parts = a.vparts > 0 ? a.vparts : 1;
    float* cw = reinterpret_cast<float*>(s_c4[w]);
    // unit g: rows [r0, r1) of volume p = g / parts
    for (int64_t g = (int64_t)blockIdx.x * kSurfWarps + w; g < a.n * parts; g += stride) {
        const int64_t p = g / parts;
        const int part = (int)(g - p * parts);
        const int r0 = nu * part / parts, r1 = nu * (part + 1) / parts;
        __syncwarp();  // the previous unit is done with s_c4 and s_y
        if (USTAGE == VOL_U_CORES) {
            cw[lane] = load_elem(a.ctrl, a.dtype, p * 64 + lane);
            cw[32 + lane] = load_elem(a.ctrl, a.dtype, p * 64 + 32 + lane);
            __syncwarp();
        }
        // Y[a][j] (a float4 over l) for rows a of the unit: entry e = 4 (a - r0) + j
        for (int e = lane; e < (r1 - r0) * 4; e += 32) {
            const int ai = r0 + (e >> 2), j = e & 3;
            float4 y;
            if (USTAGE == VOL_U_CORES) {
                const float4 bu = s_bu[ai];
                const float4 c0 = s_c4[w][j], c1 = s_c4[w][4 + j], c2 = s_c4[w][8 + j], c3 = s_c4[w][12 + j];
                y.x = fmaf(bu.w, c3.x, fmaf(bu.z, c2.x, fmaf(bu.y, c1.x, bu.x * c0.x)));
                y.y = fmaf(bu.w, c3.y, fmaf(bu.z, c2.y, fmaf(bu.y, c1.y, bu.x * c0.y)));
                y.z = fmaf(bu.w, c3.z, fmaf(bu.z, c2.z, fmaf(bu.y, c1.z, bu.x * c0.z)));
                y.w = fmaf(bu.w, c3.w, fmaf(bu.z, c2.w, fmaf(bu.y, c1.w, bu.x * c0.w)));
            } else {
                // tile q = 4 p + j at texel (2 (q mod tw), 2 (q div tw)), centres at + 0.5
                const int64_t q = p * 4 + j;
                const float u = nu > 1 ? __fdiv_rn((float)ai, (float)(nu - 1)) : 0.f;
                if (USTAGE == VOL_U_TEX_SEILER) {
                    y = seiler_tile_read(ta, q, u);
                } else {
                    const float x = (float)((int)(q % ta.tw) * 2) + 0.5f, yb = (float)((int)(q / ta.tw) * 2) + 0.5f;
                    y = tex3D<float4>(ta.tex, x + u, yb + u, 0.5f + u);
                }
                if (ta.rescale) y = ta_rescale(ta, q, y);
            }
            s_y[w][e] = y;
        }
        __syncwarp();
        float4* out = reinterpret_cast<float4*>(a.out + p * pts);
        for (int ai = r0; ai < r1; ++ai) {
            const float4* ya = s_y[w] + 4 * (ai - r0);
            const float4 y0 = ya[0], y1 = ya[1], y2 = ya[2], y3 = ya[3];
            float4* o = out + (int64_t)ai * slab4;
            for (int f = lane; f < slab4; f += 32) {
                const int b = f / q4, c0 = (f - b * q4) * 4;
                const float4 bv = s_bv[b];
                float4 z;  // Z[a][b][l], l = 0..3
                z.x = fmaf(bv.w, y3.x, fmaf(bv.z, y2.x, fmaf(bv.y, y1.x, bv.x * y0.x)));
                z.y = fmaf(bv.w, y3.y, fmaf(bv.z, y2.y, fmaf(bv.y, y1.y, bv.x * y0.y)));
                z.z = fmaf(bv.w, y3.z, fmaf(bv.z, y2.z, fmaf(bv.y, y1.z, bv.x * y0.z)));
                z.w = fmaf(bv.w, y3.w, fmaf(bv.z, y2.w, fmaf(bv.y, y1.w, bv.x * y0.w)));
                float r[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const float4 bw = s_bw[c0 + m];
                    r[m] = fmaf(bw.w, z.w, fmaf(bw.z, z.z, fmaf(bw.y, z.y, bw.x * z.x)));
                }
                o[f] = make_float4(r[0], r[1], r[2], r[3]);
            }
        }
    }
}

}  // namespace bez
