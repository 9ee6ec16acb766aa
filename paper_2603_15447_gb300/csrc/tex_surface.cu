// tex_surface.cu -- bicubic surfaces through the texture unit (paper Sec. 2.2:
// a 2x2x2 RGBA de Casteljau tile holds four cubics, one per channel).
//
// For coordinate k of patch p the tile stores the four column curves
// C[.][j][k], j = 0..3, one per channel: texel(x,y,z) channel j =
// C[x+y+z][j][k].  One trilinear read at (u,u,u) then returns the four
// isoline control points X[j][k] = sum_i B_i(u) C[i][j][k] of grid row u
// (the Sec. 2 cubic tile, four curves at once), and the cubic in v runs on
// the FP32 pipes: P[u][v][k] = sum_j B_j(v) X[j][k].  The read happens once
// per grid row and coordinate and is shared by the nv points of the row.
//
// Seiler form (Sec. 4, applied per channel; surfaces are left as future work
// in Sec. 6): the same four column cubics in the 2x2 cubic Seiler layout of a
// 2D atlas, read bilinearly at (u, u (1 - u)); two filtered axes instead of
// three, and a 2D fetch rate.
//
// Layout: tile q = p * dim + k sits at texel (2 (q mod tw), 2 (q div tw), 0)
// of a float4 (or half4) 3D atlas of depth 2; coordinates are unnormalised
// with texel centres at i + 0.5, so row u reads at (x0+0.5+u, y0+0.5+u,
// 0.5+u) and u = 0, 1 land on texel centres (exact corners).
#include "tensor_common.cuh"

namespace bez {

static_assert(kSurfTexMaxRows == kSurfMaxRows, "row limit of the texture surface kernel");

struct SurfTexArgs {
    cudaTextureObject_t tex;
    int tw;  // tiles per atlas row
};

__device__ __forceinline__ void put3(cudaSurfaceObject_t s, int fmt, int x, int y, int z, float4 v)
{
    if (fmt == 0) {
        surf3Dwrite(v, s, x * 16, y, z);
    } else {
        const __half2 lo = __floats2half2_rn(v.x, v.y), hi = __floats2half2_rn(v.z, v.w);
        surf3Dwrite(make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi)), s,
                    x * 8, y, z);
    }
}

__device__ __forceinline__ void put2(cudaSurfaceObject_t s, int fmt, int x, int y, float4 v)
{
    if (fmt == 0) {
        surf2Dwrite(v, s, x * 16, y);
    } else {
        const __half2 lo = __floats2half2_rn(v.x, v.y), hi = __floats2half2_rn(v.z, v.w);
        surf2Dwrite(make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi)), s,
                    x * 8, y);
    }
}

// one thread per tile (patch, coordinate).  SEILER: the 2x2 cubic Seiler
// layout (Sec. 4) of each column curve in its channel, [[b0, b3],
// [b0 + d1, b3 + d2]] with d1 = 3 (b1 - b0) - (b3 - b0) and
// d2 = 3 (b2 - b3) - (b0 - b3), read bilinearly at (u, u (1 - u)).
template <bool SEILER>
__global__ void k_pack_surface(const TensorArgs a, int tw, cudaSurfaceObject_t surf, int fmt)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int dim = a.dim;
    if (q >= a.n * dim) return;
    const int64_t p = q / dim;
    const int k = (int)(q - p * dim);
    const int x0 = (int)(q % tw) * 2, y0 = (int)(q / tw) * 2;
    float4 b[4];  // b[i] = (C[i][0][k], C[i][1][k], C[i][2][k], C[i][3][k])
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t base = ((p * 4 + i) * 4) * dim + k;
        b[i] = make_float4(load_elem(a.ctrl, a.dtype, base), load_elem(a.ctrl, a.dtype, base + dim),
                           load_elem(a.ctrl, a.dtype, base + 2 * dim), load_elem(a.ctrl, a.dtype, base + 3 * dim));
    }
    if (SEILER) {
        const float4 d1 = make_float4(3.f * (b[1].x - b[0].x) - (b[3].x - b[0].x), 3.f * (b[1].y - b[0].y) - (b[3].y - b[0].y),
                                      3.f * (b[1].z - b[0].z) - (b[3].z - b[0].z), 3.f * (b[1].w - b[0].w) - (b[3].w - b[0].w));
        const float4 d2 = make_float4(3.f * (b[2].x - b[3].x) - (b[0].x - b[3].x), 3.f * (b[2].y - b[3].y) - (b[0].y - b[3].y),
                                      3.f * (b[2].z - b[3].z) - (b[0].z - b[3].z), 3.f * (b[2].w - b[3].w) - (b[0].w - b[3].w));
        put2(surf, fmt, x0, y0, b[0]);
        put2(surf, fmt, x0 + 1, y0, b[3]);
        put2(surf, fmt, x0, y0 + 1, make_float4(b[0].x + d1.x, b[0].y + d1.y, b[0].z + d1.z, b[0].w + d1.w));
        put2(surf, fmt, x0 + 1, y0 + 1, make_float4(b[3].x + d2.x, b[3].y + d2.y, b[3].z + d2.z, b[3].w + d2.w));
        return;
    }
#pragma unroll
    for (int z = 0; z < 2; ++z)
#pragma unroll
        for (int y = 0; y < 2; ++y)
#pragma unroll
            for (int x = 0; x < 2; ++x) put3(surf, fmt, x0 + x, y0 + y, z, b[x + y + z]);
}

// One warp per patch: lanes read the isoline control points of their rows,
// then the warp sweeps the grid a row segment of up to 32 points at a time
// and stores it through a warp-private staging buffer as consecutive floats.
template <int DIM, bool SEILER>
__global__ void __launch_bounds__(kSurfWarps * 32, 4) k_surface_tex(const TensorArgs a, const SurfTexArgs ta)
{
    __shared__ float4 s_bv[kTensorMaxGrid];                   // Bv[b][0..3]
    __shared__ float4 s_x[kSurfWarps][kSurfMaxRows * DIM];    // X[row][k] over j
    __shared__ float s_st[kSurfWarps][32 * DIM];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    bernstein_table(reinterpret_cast<float*>(s_bv), a.nv, 3, tid, kSurfWarps * 32);
    __syncthreads();

    const int nu = a.nu, nv = a.nv;
    const int64_t pts = (int64_t)nu * nv;
    const int64_t stride = (int64_t)gridDim.x * kSurfWarps;
    float* st = s_st[w];
    for (int64_t p = (int64_t)blockIdx.x * kSurfWarps + w; p < a.n; p += stride) {
        __syncwarp();  // the previous patch is done with s_x
        for (int row = lane; row < nu; row += 32) {
            const float u = nu > 1 ? __fdiv_rn((float)row, (float)(nu - 1)) : 0.f;
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                const int64_t q = p * DIM + k;
                const float x = (float)((int)(q % ta.tw) * 2) + 0.5f, y = (float)((int)(q / ta.tw) * 2) + 0.5f;
                s_x[w][row * DIM + k] = SEILER ? tex2D<float4>(ta.tex, x + u, y + fmaf(-u, u, u))
                                               : tex3D<float4>(ta.tex, x + u, y + u, 0.5f + u);
            }
        }
        __syncwarp();
        float* out = a.out + p * pts * DIM;
        for (int b0 = 0; b0 < nv; b0 += 32) {
            const int b = b0 + lane;
            const float4 bv = b < nv ? s_bv[b] : make_float4(0.f, 0.f, 0.f, 0.f);
            const int valid = min(32, nv - b0) * DIM;
            for (int row = 0; row < nu; ++row) {
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    const float4 X = s_x[w][row * DIM + k];
                    st[lane * DIM + k] = fmaf(bv.w, X.w, fmaf(bv.z, X.z, fmaf(bv.y, X.y, bv.x * X.x)));
                }
                __syncwarp();
                float* o = out + ((int64_t)row * nv + b0) * DIM;
#pragma unroll
                for (int m = 0; m < DIM; ++m) {
                    const int idx = lane + 32 * m;
                    if (idx < valid) o[idx] = st[idx];
                }
                __syncwarp();
            }
        }
    }
}

// tiles per atlas row: a power of two near sqrt(tiles) so the atlas is
// roughly square (small coordinates keep more fractional bits)
static int surface_tiles_per_row(int64_t tiles, int max_w)
{
    int tw = 1;
    while ((int64_t)tw * tw < tiles && tw * 4 <= max_w) tw *= 2;
    return tw;
}

LaunchResult launch_tex_surface(const TensorLaunch& t, bool seiler, TexState& ts, cudaStream_t s,
                                const LaunchHooks& h)
{
    TensorArgs a{};
    a.ctrl = t.ctrl;
    a.dtype = t.dtype;
    a.n = t.n;
    a.du = t.du;
    a.dv = t.dv;
    a.dw = t.dw;
    a.dim = t.dim;
    a.nu = t.nu;
    a.nv = t.nv;
    a.nw = t.nw;
    a.out = t.out;
    const int64_t tiles = a.n * a.dim;
    const int tw = surface_tiles_per_row(tiles, ts.max3d);
    const int64_t rows = (tiles + tw - 1) / tw;
    if (rows * 2 > ts.max3d) return {0, cudaErrorInvalidValue};
    const int fmt = a.dtype == 1 ? 1 : 0;
    Atlas& at = seiler ? ts.surf2 : ts.surf3;
    cudaError_t e = atlas_ensure(at, tw * 2, (int)(rows * 2), seiler ? 0 : 2, fmt);
    if (e != cudaSuccess) return {0, e};
    h.count(h.self);
    if (seiler) k_pack_surface<true><<<(unsigned)((tiles + 255) / 256), 256, 0, s>>>(a, tw, at.surf, fmt);
    else k_pack_surface<false><<<(unsigned)((tiles + 255) / 256), 256, 0, s>>>(a, tw, at.surf, fmt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return {1, e};
    const void* kern;
    if (seiler)
        kern = a.dim == 1   ? (const void*)k_surface_tex<1, true>
               : a.dim == 2 ? (const void*)k_surface_tex<2, true>
               : a.dim == 3 ? (const void*)k_surface_tex<3, true>
                            : (const void*)k_surface_tex<4, true>;
    else
        kern = a.dim == 1   ? (const void*)k_surface_tex<1, false>
               : a.dim == 2 ? (const void*)k_surface_tex<2, false>
               : a.dim == 3 ? (const void*)k_surface_tex<3, false>
                            : (const void*)k_surface_tex<4, false>;
    const int grid = persistent_grid(kern, kSurfWarps * 32, 0, h.sm_count, (a.n + kSurfWarps - 1) / kSurfWarps);
    SurfTexArgs sa{at.tex, tw};
    void* args[] = {(void*)&a, (void*)&sa};
    h.count(h.self);
    h.begin(h.self, s);
    e = cudaLaunchKernel(kern, dim3(grid), dim3(kSurfWarps * 32), args, 0, s);
    h.end(h.self, s);
    return {2, e};
}

}  // namespace bez
