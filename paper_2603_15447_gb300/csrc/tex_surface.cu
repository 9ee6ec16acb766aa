// tex_surface.cu -- bicubic surfaces and tricubic scalar volumes through the
// texture unit (paper Sec. 2.2: a 2x2x2 RGBA de Casteljau tile holds four
// cubics, one per channel).
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
// Tricubic scalar volumes (Sec. 6 leaves volumes as future work) take the
// same tiles one axis up: tile q = 4 p + j holds the u cubics C[.][j][l],
// l = 0..3, one per channel, so one read per (row u, j) gives Y[u][j][.],
// and v and w contract on the FP32 pipes (k_volume_tricubic1_warp).
//
// Spread Seiler tiles (tex_spread s >= 2): each channel's Seiler bilinear
// function F(X, Y) = L(b0 + (Y/4) d1, b3 + (Y/4) d2, X) sampled on an
// (s+1) x (s+1) texel grid and read at (s u, 4 s u (1 - u)); the 8-bit
// filter-weight rounding then moves the read s times less (tex.cu).
//
// Layout: surface tile q = p * dim + k sits at texel (2 (q mod tw),
// 2 (q div tw), 0) of a float4, half4 or unorm 3D atlas of depth 2 (2D for
// Seiler tiles, (s+1) texels per tile axis when spread); coordinates are
// unnormalised with texel centres at i + 0.5, so row u reads at
// (x0+0.5+u, y0+0.5+u, 0.5+u) and u = 0, 1 land on texel centres (exact
// corners).
#include "tensor_common.cuh"
#include "texel.cuh"

namespace bez {

static_assert(kSurfTexMaxRows == kSurfMaxRows, "row limit of the texture surface kernel");
static_assert(kVolTexMaxRows == kVolMaxRows, "row limit of the texture volume kernel");

// One thread per tile: four u cubics, one per channel.  Surface tile
// q = p dim + k holds the column cubics C[.][j][k] (channel j); volume tile
// q = 4 p + j (scalar volumes) holds C[.][j][l] (channel l).  SEILER: the
// 2x2 cubic Seiler layout (Sec. 4) of each cubic in its channel, [[b0, b3],
// [b0 + d1, b3 + d2]] with d1 = 3 (b1 - b0) - (b3 - b0) and
// d2 = 3 (b2 - b3) - (b0 - b3), read bilinearly at (u, u (1 - u)).
// unorm formats: each tile's texels are stored as lo + scale u per channel
// (rescale[2q], rescale[2q + 1]).
template <bool SEILER>
__global__ void k_pack_surface(const TensorArgs a, int tw, cudaSurfaceObject_t surf, int fmt, float4* rescale)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool vol = a.dw >= 0;
    const int dim = a.dim;
    const int per = vol ? 4 : dim;  // tiles per patch / volume
    if (q >= a.n * per) return;
    const int64_t p = q / per;
    const int r = (int)(q - p * per);
    const int x0 = (int)(q % tw) * 2, y0 = (int)(q / tw) * 2;
    // b[i] = the four cubics' control point i: C[i][0..3][r] (surface) or C[i][r][0..3] (volume)
    const int cs = vol ? 1 : dim;   // channel stride in elements
    float4 b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t base = vol ? ((p * 4 + i) * 4 + r) * 4 : ((p * 4 + i) * 4) * dim + r;
        b[i] = make_float4(load_elem(a.ctrl, a.dtype, base), load_elem(a.ctrl, a.dtype, base + cs),
                           load_elem(a.ctrl, a.dtype, base + 2 * cs), load_elem(a.ctrl, a.dtype, base + 3 * cs));
    }
    // the tile's distinct texel values: the four control points (de Casteljau
    // tile: texel(x,y,z) = b[x+y+z]) or the four Seiler corners
    float4 v[4];
    if (SEILER) {
        const float4 d1 = make_float4(3.f * (b[1].x - b[0].x) - (b[3].x - b[0].x), 3.f * (b[1].y - b[0].y) - (b[3].y - b[0].y),
                                      3.f * (b[1].z - b[0].z) - (b[3].z - b[0].z), 3.f * (b[1].w - b[0].w) - (b[3].w - b[0].w));
        const float4 d2 = make_float4(3.f * (b[2].x - b[3].x) - (b[0].x - b[3].x), 3.f * (b[2].y - b[3].y) - (b[0].y - b[3].y),
                                      3.f * (b[2].z - b[3].z) - (b[0].z - b[3].z), 3.f * (b[2].w - b[3].w) - (b[0].w - b[3].w));
        v[0] = b[0];
        v[1] = b[3];
        v[2] = make_float4(b[0].x + d1.x, b[0].y + d1.y, b[0].z + d1.z, b[0].w + d1.w);
        v[3] = make_float4(b[3].x + d2.x, b[3].y + d2.y, b[3].z + d2.z, b[3].w + d2.w);
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = b[i];
    }
    if (fmt >= TEXEL_UNORM16) {
        // per channel: lo + scale u, u in [0, 1], over the tile's values; a
        // constant channel maps to code 0 (scale 1 avoids dividing by 0)
        float4 lo = v[0], hi = v[0];
#pragma unroll
        for (int i = 1; i < 4; ++i) {
            lo = min4(lo, v[i]);
            hi = max4(hi, v[i]);
        }
        float4 sc = make_float4(hi.x - lo.x, hi.y - lo.y, hi.z - lo.z, hi.w - lo.w);
        sc = make_float4(sc.x > 0.f ? sc.x : 1.f, sc.y > 0.f ? sc.y : 1.f, sc.z > 0.f ? sc.z : 1.f, sc.w > 0.f ? sc.w : 1.f);
        rescale[2 * q] = lo;
        rescale[2 * q + 1] = sc;
#pragma unroll
        for (int i = 0; i < 4; ++i)
            v[i] = make_float4(__fdiv_rn(v[i].x - lo.x, sc.x), __fdiv_rn(v[i].y - lo.y, sc.y),
                               __fdiv_rn(v[i].z - lo.z, sc.z), __fdiv_rn(v[i].w - lo.w, sc.w));
    }
    if constexpr (SEILER) {
        put(surf, fmt, x0, y0, 0, false, v[0]);
        put(surf, fmt, x0 + 1, y0, 0, false, v[1]);
        put(surf, fmt, x0, y0 + 1, 0, false, v[2]);
        put(surf, fmt, x0 + 1, y0 + 1, 0, false, v[3]);
    } else {
#pragma unroll
        for (int z = 0; z < 2; ++z)
#pragma unroll
            for (int y = 0; y < 2; ++y)
#pragma unroll
                for (int x = 0; x < 2; ++x) put(surf, fmt, x0 + x, y0 + y, z, true, v[x + y + z]);
    }
}

// Spread Seiler tiles: one thread per texel (tile q, row j, column i).
__global__ void k_pack_surface_spread(const TensorArgs a, int tw, int sp, cudaSurfaceObject_t surf, int fmt,
                                      float4* rescale)
{
    const int n1 = sp + 1;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool vol = a.dw >= 0;
    const int dim = a.dim;
    const int per = vol ? 4 : dim;
    const int64_t q = idx / (n1 * n1);
    if (q >= a.n * per) return;
    const int rr = (int)(idx - q * n1 * n1);
    const int jj = rr / n1, ii = rr - jj * n1;
    const int64_t p = q / per;
    const int r = (int)(q - p * per);
    const int cs = vol ? 1 : dim;
    float4 b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t base = vol ? ((p * 4 + i) * 4 + r) * 4 : ((p * 4 + i) * 4) * dim + r;
        b[i] = make_float4(load_elem(a.ctrl, a.dtype, base), load_elem(a.ctrl, a.dtype, base + cs),
                           load_elem(a.ctrl, a.dtype, base + 2 * cs), load_elem(a.ctrl, a.dtype, base + 3 * cs));
    }
    // d1 = 3 (b1 - b0) - (b3 - b0), d2 = 3 (b2 - b3) - (b0 - b3) per channel (Sec. 3.1)
    auto comb = [](float4 x0, float4 x1, float4 x3) {
        return make_float4(3.f * (x1.x - x0.x) - (x3.x - x0.x), 3.f * (x1.y - x0.y) - (x3.y - x0.y),
                           3.f * (x1.z - x0.z) - (x3.z - x0.z), 3.f * (x1.w - x0.w) - (x3.w - x0.w));
    };
    const float4 d1 = comb(b[0], b[1], b[3]), d2 = comb(b[3], b[2], b[0]);
    const float inv = 1.f / (float)sp;  // sp a power of two: exact
    auto texel = [&](int x, int y) {
        const float ys = 0.25f * inv * (float)y, xs = inv * (float)x;
        const float4 lo = make_float4(b[0].x + ys * d1.x, b[0].y + ys * d1.y, b[0].z + ys * d1.z, b[0].w + ys * d1.w);
        const float4 hi = make_float4(b[3].x + ys * d2.x, b[3].y + ys * d2.y, b[3].z + ys * d2.z, b[3].w + ys * d2.w);
        const float xl = 1.f - xs;
        return make_float4(xl * lo.x + xs * hi.x, xl * lo.y + xs * hi.y, xl * lo.z + xs * hi.z, xl * lo.w + xs * hi.w);
    };
    float4 v = texel(ii, jj);
    if (fmt >= TEXEL_UNORM16) {
        // per channel over the tile's values: a bilinear function takes its extremes at the corners
        const float4 c00 = texel(0, 0), c10 = texel(sp, 0), c01 = texel(0, sp), c11 = texel(sp, sp);
        const float4 lo = min4(min4(c00, c10), min4(c01, c11)), hi = max4(max4(c00, c10), max4(c01, c11));
        float4 sc = make_float4(hi.x - lo.x, hi.y - lo.y, hi.z - lo.z, hi.w - lo.w);
        sc = make_float4(sc.x > 0.f ? sc.x : 1.f, sc.y > 0.f ? sc.y : 1.f, sc.z > 0.f ? sc.z : 1.f, sc.w > 0.f ? sc.w : 1.f);
        if (ii == 0 && jj == 0) {
            rescale[2 * q] = lo;
            rescale[2 * q + 1] = sc;
        }
        v = make_float4(__fdiv_rn(v.x - lo.x, sc.x), __fdiv_rn(v.y - lo.y, sc.y), __fdiv_rn(v.z - lo.z, sc.z),
                        __fdiv_rn(v.w - lo.w, sc.w));
    }
    put(surf, fmt, (int)(q % tw) * n1 + ii, (int)(q / tw) * n1 + jj, 0, false, v);
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
    // the filtered reads of grid row `row` of patch pp, one per coordinate
    auto fetch = [&](int64_t pp, int row, float4 (&X)[DIM]) {
        const float u = nu > 1 ? __fdiv_rn((float)row, (float)(nu - 1)) : 0.f;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const int64_t q = pp * DIM + k;
            if (SEILER) {
                X[k] = seiler_tile_read(ta, q, u);
            } else {
                const float x = (float)((int)(q % ta.tw) * 2) + 0.5f, y = (float)((int)(q / ta.tw) * 2) + 0.5f;
                X[k] = tex3D<float4>(ta.tex, x + u, y + u, 0.5f + u);
            }
            if (ta.rescale) X[k] = ta_rescale(ta, q, X[k]);
        }
    };
    // With at most 32 rows a lane owns one row, and the reads of the warp's
    // next patch are issued before the current patch's sweep, so their
    // latency overlaps the stores.
    const bool one_row = nu <= 32;
    int64_t p = (int64_t)blockIdx.x * kSurfWarps + w;
    float4 Xn[DIM];
    if (one_row && p < a.n && lane < nu) fetch(p, lane, Xn);
    for (; p < a.n; p += stride) {
        __syncwarp();  // the previous patch is done with s_x
        if (one_row) {
            if (lane < nu) {
#pragma unroll
                for (int k = 0; k < DIM; ++k) s_x[w][lane * DIM + k] = Xn[k];
                if (p + stride < a.n) fetch(p + stride, lane, Xn);
            }
        } else {
            for (int row = lane; row < nu; row += 32) {
                float4 X[DIM];
                fetch(p, row, X);
#pragma unroll
                for (int k = 0; k < DIM; ++k) s_x[w][row * DIM + k] = X[k];
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

// tiles per atlas row: a power of two near sqrt(tiles) so the atlas of
// n1 x n1 tiles is roughly square (small coordinates keep more fractional
// bits)
static int surface_tiles_per_row(int64_t tiles, int max_w, int n1)
{
    int tw = 1;
    while ((int64_t)tw * tw < tiles && tw * 2 * n1 <= max_w) tw *= 2;
    return tw;
}

LaunchResult launch_tex_surface(const TensorLaunch& t, bool seiler, int tex_format, int spread, TexState& ts,
                                cudaStream_t s, const LaunchHooks& h)
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
    const bool vol = a.dw >= 0;
    const int64_t tiles = a.n * (vol ? 4 : a.dim);
    const int sp = seiler && spread > 1 ? spread : 1;
    const int n1 = sp + 1;
    const int tw = surface_tiles_per_row(tiles, ts.max3d, n1);
    const int64_t rows = (tiles + tw - 1) / tw;
    if (rows * n1 > ts.max3d) return {0, cudaErrorInvalidValue};
    const int fmt = texel_format(a.dtype, tex_format);
    Atlas& at = seiler ? ts.surf2 : ts.surf3;
    cudaError_t e = atlas_ensure(at, tw * n1, (int)(rows * n1), seiler ? 0 : 2, fmt);
    if (e != cudaSuccess) return {0, e};
    float4* rs = nullptr;
    if ((e = rescale_buffer(ts, fmt, tiles, &rs)) != cudaSuccess) return {0, e};
    h.count(h.self);
    if (sp > 1) {
        const int64_t n_texels = tiles * n1 * n1;
        k_pack_surface_spread<<<(unsigned)((n_texels + 255) / 256), 256, 0, s>>>(a, tw, sp, at.surf, fmt, rs);
    } else if (seiler) {
        k_pack_surface<true><<<(unsigned)((tiles + 255) / 256), 256, 0, s>>>(a, tw, at.surf, fmt, rs);
    } else {
        k_pack_surface<false><<<(unsigned)((tiles + 255) / 256), 256, 0, s>>>(a, tw, at.surf, fmt, rs);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return {1, e};
    const void* kern;
    if (vol)
        kern = seiler ? (const void*)k_volume_tricubic1_warp<VOL_U_TEX_SEILER>
                      : (const void*)k_volume_tricubic1_warp<VOL_U_TEX_DC>;
    else if (seiler)
        kern = a.dim == 1   ? (const void*)k_surface_tex<1, true>
               : a.dim == 2 ? (const void*)k_surface_tex<2, true>
               : a.dim == 3 ? (const void*)k_surface_tex<3, true>
                            : (const void*)k_surface_tex<4, true>;
    else
        kern = a.dim == 1   ? (const void*)k_surface_tex<1, false>
               : a.dim == 2 ? (const void*)k_surface_tex<2, false>
               : a.dim == 3 ? (const void*)k_surface_tex<3, false>
                            : (const void*)k_surface_tex<4, false>;
    a.vparts = vol ? volume_parts(a.n, a.nu, h.sm_count) : 1;
    const int grid = persistent_grid(kern, kSurfWarps * 32, 0, h.sm_count,
                                     (a.n * a.vparts + kSurfWarps - 1) / kSurfWarps);
    SurfTexArgs sa{at.tex, tw, rs, sp};
    void* args[] = {(void*)&a, (void*)&sa};
    h.count(h.self);
    h.begin(h.self, s);
    e = cudaLaunchKernel(kern, dim3(grid), dim3(kSurfWarps * 32), args, 0, s);
    h.end(h.self, s);
    return {2, e};
}

}  // namespace bez
