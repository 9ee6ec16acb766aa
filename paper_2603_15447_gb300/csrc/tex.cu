// tex.cu -- texture-path curve evaluators (paper Sec. 2 and Sec. 4).
//
// Control points are packed by a surface-write kernel into cudaArray atlases
// owned by the context, then read with hardware linear filtering:
//
//   DC3   cubic, one 2x2x2 tile, texel(x,y,z) = b_(x+y+z), one trilinear read
//         at (t, t, t): front slice is the quadratic (b0,b1,b2), back slice
//         (b1,b2,b3) (Sec. 2).
//   DCN   any other degree: strip texel(x,y,z) = b_(x+y+z), x in [0, d-2];
//         window i read at (i+t, t, t) gives the level-3 de Casteljau point
//         of b_i..b_(i+3); the remaining d-3 levels are FP32 lerps (Sec. 2:
//         "further interpolation levels can be done in the shader").
//         Degrees 1, 2 read one tile with the unused axes at texel centres.
//   HYB3  cubic hybrid (Fig. 3): 2D strip texel(x,y) = b_(x+y); two bilinear
//         reads give the quadratics (b0,b1,b2), (b1,b2,b3); final lerp in FP32.
//   HYBN  the same 2D strip for other degrees: d-1 bilinear reads, d-2 lerps.
//   SEIL2 degrees 2, 3: 2x2 tile [[b0, bd], [b0+d1, bd+d_(d-1)]] read at
//         (t, st) (Sec. 4, Eq. 6 and the layout table).
//   SEIL3 degrees 4, 5: 2x2x2 tile, z=0 [[b0,bd],[b0,bd]],
//         z=1 [[b0+d1, bd+d_(d-1)], [b0+d1+d2, bd+d_(d-1)+d_(d-2)]] read at
//         (t, st, st) (Sec. 4, Eq. 7 and the layout table).
//   SEIL3Q degrees 6, 7 (beyond the layout table; Sec. 6 leaves them open):
//         trilinear filtering of a 2x2x2 tile at (x, y, z) is
//         L0(x) + y L1(x) + z L2(x) + yz L3(x) with L_k linear in x, so reading
//         at (t, 4 st, 16 st^2) a tile holding L0 = L(d0, dd), L1/4, L2/16 and
//         L3/64 in its corners gives the Seiler form L0 + st L1 + st^2 L2 +
//         st^3 L3 of any degree <= 7 (L_k = L(d_k, d_(d-k), t)).  The 4 and 16
//         use the whole weight range of the y and z axes; d_k come from the
//         exact peeling of the s-power form in FP64.
//   SEIL2S degrees 2, 3 with a spread s >= 2: the SEIL2 tile's bilinear
//         function F(x, y) = L(b0, bd, x) + (y/4) L(d1, d_(d-1), x), y = 4 st,
//         sampled on an (s+1) x (s+1) texel grid (texel (i, j) = F(i/s, j/s))
//         and read at (s t, 4 s st).  Bilinear filtering of a finer grid of a
//         bilinear function reproduces the function, so the read computes the
//         same Seiler form, but the 8-bit filter weights (Sec. 2.3) now
//         quantise a coordinate s times finer: the hardware forms the weights
//         of a cell from its fractions rounded to 1/256 (the twist weight
//         round8(a b)), so every rounding term of a read shrinks by s (the
//         twist term by s^2) at (s+1)^2 / 4 times the texture memory.
//
// Coordinates are unnormalised with texel centres at i + 0.5, so the paper's
// [0.25, 0.75] remap of a 2-texel axis becomes x = x0 + 0.5 + t; for the st
// axis the offset is added after the product (Sec. 4).  Addressing clamps.
#include "curve_eval.cuh"
#include "texel.cuh"

namespace bez {

enum { TK_DC3 = 0, TK_DCN = 1, TK_HYB3 = 2, TK_HYBN = 3, TK_SEIL2 = 4, TK_SEIL3 = 5, TK_SEIL3Q = 6, TK_SEIL2S = 7 };

struct TexArgs {
    cudaTextureObject_t tex;
    int tw;   // tiles per atlas row
    int wt;   // tile width in texels
    int deg;
    float4* rescale;  // unorm formats: per curve (offset, scale) of its tile; nullptr for float / half texels
    int ht;   // tile height in texels
    int sp;   // SEIL2S: texel intervals per tile axis (spread)
};

// ---------------------------------------------------------------- atlases (host)

void atlas_free(Atlas& at)
{
    if (at.tex) cudaDestroyTextureObject(at.tex);
    if (at.surf) cudaDestroySurfaceObject(at.surf);
    if (at.arr) cudaFreeArray(at.arr);
    at = Atlas{};
}

cudaError_t atlas_ensure(Atlas& at, int w, int h, int depth, int fmt)
{
    if (at.arr && at.depth == depth && at.fmt == fmt && at.w >= w && at.h >= h) return cudaSuccess;
    if (at.arr && at.depth == depth && at.fmt == fmt) {
        w = w > at.w ? w : at.w;
        h = h > at.h ? h : at.h;
    }
    if (at.arr) {
        cudaError_t e = cudaDeviceSynchronize();  // the old atlas may still be read
        if (e != cudaSuccess) return e;
        atlas_free(at);
    }
    // fmt 0 float4, 1 half4, 2 unorm16 x 4, 3 unorm8 x 4 (read as normalised floats)
    cudaChannelFormatDesc cd = fmt == 0   ? cudaCreateChannelDesc<float4>()
                               : fmt == 1 ? cudaCreateChannelDescHalf4()
                               : fmt == 2 ? cudaCreateChannelDesc<ushort4>()
                                          : cudaCreateChannelDesc<uchar4>();
    cudaError_t e;
    if (depth > 0) e = cudaMalloc3DArray(&at.arr, &cd, make_cudaExtent(w, h, depth), cudaArraySurfaceLoadStore);
    else e = cudaMallocArray(&at.arr, &cd, w, h, cudaArraySurfaceLoadStore);
    if (e != cudaSuccess) {
        at.arr = nullptr;
        return e;
    }
    cudaResourceDesc rd = {};
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = at.arr;
    cudaTextureDesc td = {};
    td.addressMode[0] = td.addressMode[1] = td.addressMode[2] = cudaAddressModeClamp;
    td.filterMode = cudaFilterModeLinear;
    td.readMode = fmt >= 2 ? cudaReadModeNormalizedFloat : cudaReadModeElementType;
    td.normalizedCoords = 0;
    e = cudaCreateTextureObject(&at.tex, &rd, &td, nullptr);
    if (e == cudaSuccess) e = cudaCreateSurfaceObject(&at.surf, &rd);
    if (e != cudaSuccess) {
        atlas_free(at);
        return e;
    }
    at.w = w;
    at.h = h;
    at.depth = depth;
    at.fmt = fmt;
    return cudaSuccess;
}

// ---------------------------------------------------------------- packers

__device__ __forceinline__ float4 add4(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ float4 sub4(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
__device__ __forceinline__ float4 scale4(float s, float4 a) { return make_float4(s * a.x, s * a.y, s * a.z, s * a.w); }

// Seiler difference terms by the closed forms of Sec. 3.1 (degree 2..5):
// d1 = d(b1-b0) - (bd-b0), d_(d-1) = d(b_(d-1)-bd) - (b0-bd), and for d = 4, 5
// d2 = C(d,2)(b2-b1) - C(d-2,2)(b1-b0) - (d-3)(b_(d-1)-bd) - 3(b_(d-1)-b1),
// d_(d-2) mirrored.
__device__ void seiler_terms(const float4* b, int d, float4& d1, float4& dl, float4& d2, float4& dl2)
{
    const float fd = (float)d;
    d1 = sub4(scale4(fd, sub4(b[1], b[0])), sub4(b[d], b[0]));
    dl = sub4(scale4(fd, sub4(b[d - 1], b[d])), sub4(b[0], b[d]));
    d2 = dl2 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (d >= 4) {
        const float c2 = (float)(d * (d - 1) / 2), c2m = (float)((d - 2) * (d - 3) / 2), e = (float)(d - 3);
        d2 = sub4(sub4(sub4(scale4(c2, sub4(b[2], b[1])), scale4(c2m, sub4(b[1], b[0]))),
                       scale4(e, sub4(b[d - 1], b[d]))),
                  scale4(3.f, sub4(b[d - 1], b[1])));
        dl2 = sub4(sub4(sub4(scale4(c2, sub4(b[d - 2], b[d - 1])), scale4(c2m, sub4(b[d - 1], b[d]))),
                        scale4(e, sub4(b[1], b[0]))),
                   scale4(3.f, sub4(b[1], b[d - 1])));
    }
}

// Seiler terms of degree 6 or 7 by peeling P = L(P(0), P(1), t) + t(1-t) Q
// in the Bernstein basis (FP64): lo[k] = d_k, hi[k] = d_(d-k), k = 0..3
// (d_0 = b_0, d_d = b_d; for d = 6, lo[3] = hi[3] = d_3).
__device__ void seiler_terms_peeled(const float4* b, int d, float4 (&lo)[4], float4 (&hi)[4])
{
    for (int k = 0; k < 4; ++k) {
        double c[8];
        for (int i = 0; i <= d; ++i) c[i] = k == 0 ? b[i].x : k == 1 ? b[i].y : k == 2 ? b[i].z : b[i].w;
        int m = d;
        for (int lvl = 0; lvl < 4; ++lvl) {
            const double c0 = c[0], cm = c[m < 0 ? 0 : m];
            float* L = k == 0 ? &lo[lvl].x : k == 1 ? &lo[lvl].y : k == 2 ? &lo[lvl].z : &lo[lvl].w;
            float* R = k == 0 ? &hi[lvl].x : k == 1 ? &hi[lvl].y : k == 2 ? &hi[lvl].z : &hi[lvl].w;
            if (m < 0) {
                *L = *R = 0.f;
                continue;
            }
            *L = (float)c0;
            *R = (float)cm;
            if (m < 2) {
                m = -1;
                continue;
            }
            const double mm = (double)m;
            for (int j = 0; j <= m - 2; ++j) {
                const double i1 = (double)(j + 1);
                const double q = (c[j + 1] - c0) - (i1 / mm) * (cm - c0);
                c[j] = q * (mm * (mm - 1.0)) / (i1 * (mm - 1.0 - (double)j));
            }
            m -= 2;
        }
    }
}


// Texels of curve c's tile: emit(x, y, z, value) for every texel.
template <int KIND, class Emit>
__device__ __forceinline__ void tile_texels(const float4* b, int d, int wt, Emit&& emit)
{
    if (KIND == TK_DC3 || KIND == TK_DCN) {
        for (int z = 0; z < 2; ++z)
            for (int y = 0; y < 2; ++y)
                for (int x = 0; x < wt; ++x) emit(x, y, z, b[min(x + y + z, d)]);
    } else if (KIND == TK_HYB3 || KIND == TK_HYBN) {
        for (int y = 0; y < 2; ++y)
            for (int x = 0; x < wt; ++x) emit(x, y, 0, b[min(x + y, d)]);
    } else if (KIND == TK_SEIL2S) {
        // wt = s + 1 texels per axis; row j holds st = j / (4 s)
        float4 d1, dl, d2, dl2;
        seiler_terms(b, d, d1, dl, d2, dl2);
        const int sp = wt - 1;
        const float inv = 1.f / (float)sp;  // s is a power of two: exact
        for (int y = 0; y <= sp; ++y) {
            const float ys = 0.25f * inv * (float)y;
            const float4 lo = add4(b[0], scale4(ys, d1)), hi = add4(b[d], scale4(ys, dl));
            for (int x = 0; x <= sp; ++x) {
                const float xs = inv * (float)x;
                emit(x, y, 0, add4(scale4(1.f - xs, lo), scale4(xs, hi)));
            }
        }
    } else if (KIND == TK_SEIL3Q) {
        float4 lo[4], hi[4];
        seiler_terms_peeled(b, d, lo, hi);
        const float4 z0y1l = add4(lo[0], scale4(0.25f, lo[1])), z0y1h = add4(hi[0], scale4(0.25f, hi[1]));
        emit(0, 0, 0, lo[0]);
        emit(1, 0, 0, hi[0]);
        emit(0, 1, 0, z0y1l);
        emit(1, 1, 0, z0y1h);
        emit(0, 0, 1, add4(lo[0], scale4(0.0625f, lo[2])));
        emit(1, 0, 1, add4(hi[0], scale4(0.0625f, hi[2])));
        emit(0, 1, 1, add4(z0y1l, add4(scale4(0.0625f, lo[2]), scale4(0.015625f, lo[3]))));
        emit(1, 1, 1, add4(z0y1h, add4(scale4(0.0625f, hi[2]), scale4(0.015625f, hi[3]))));
    } else {
        float4 d1, dl, d2, dl2;
        seiler_terms(b, d, d1, dl, d2, dl2);
        if (KIND == TK_SEIL2) {
            emit(0, 0, 0, b[0]);
            emit(1, 0, 0, b[d]);
            emit(0, 1, 0, add4(b[0], d1));
            emit(1, 1, 0, add4(b[d], dl));
        } else {
            emit(0, 0, 0, b[0]);
            emit(1, 0, 0, b[d]);
            emit(0, 1, 0, b[0]);
            emit(1, 1, 0, b[d]);
            const float4 s1 = add4(b[0], d1), s2 = add4(b[d], dl);
            emit(0, 0, 1, s1);
            emit(1, 0, 1, s2);
            emit(0, 1, 1, add4(s1, d2));
            emit(1, 1, 1, add4(s2, dl2));
        }
    }
}

// One thread per curve: its tile's texels into the atlas.  Unorm formats
// (Sec. 2.3: low-bit-depth texels hold [0, 1]) store (v - lo) / scale with
// lo and scale the tile's per-component minimum and range, recorded in
// ta.rescale for the evaluator, which maps the filtered value back by
// lo + scale * f (filtering is affine, so this commutes with it).
template <int KIND>
__global__ void k_pack(const CurveArgs a, TexArgs ta, cudaSurfaceObject_t surf, int fmt)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.n_curves) return;
    const int d = a.degree, dim = a.dim;
    float4 b[kMaxDegree + 1];
    for (int i = 0; i <= d; ++i) {
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < dim; ++k) v[k] = load_elem(a.ctrl, a.dtype, (c * (d + 1) + i) * dim + k);
        b[i] = make_float4(v[0], v[1], v[2], v[3]);
    }
    const int x0 = (int)(c % ta.tw) * ta.wt, y0 = (int)(c / ta.tw) * ta.ht;
    const bool is3d = KIND == TK_DC3 || KIND == TK_DCN || KIND == TK_SEIL3 || KIND == TK_SEIL3Q;
    if (fmt < 2) {
        tile_texels<KIND>(b, d, ta.wt, [&](int x, int y, int z, float4 v) { put(surf, fmt, x0 + x, y0 + y, z, is3d, v); });
        return;
    }
    float4 lo = make_float4(INFINITY, INFINITY, INFINITY, INFINITY), hi = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
    tile_texels<KIND>(b, d, ta.wt, [&](int, int, int, float4 v) {
        lo = min4(lo, v);
        hi = max4(hi, v);
    });
    float4 sc = sub4(hi, lo);
    // a constant component maps to code 0; its scale is irrelevant but must not divide by 0
    sc = make_float4(sc.x > 0.f ? sc.x : 1.f, sc.y > 0.f ? sc.y : 1.f, sc.z > 0.f ? sc.z : 1.f, sc.w > 0.f ? sc.w : 1.f);
    ta.rescale[2 * c] = lo;
    ta.rescale[2 * c + 1] = sc;
    tile_texels<KIND>(b, d, ta.wt, [&](int x, int y, int z, float4 v) {
        const float4 u = make_float4(__fdiv_rn(v.x - lo.x, sc.x), __fdiv_rn(v.y - lo.y, sc.y), __fdiv_rn(v.z - lo.z, sc.z),
                                     __fdiv_rn(v.w - lo.w, sc.w));
        put(surf, fmt, x0 + x, y0 + y, z, is3d, u);
    });
}

// Spread Seiler tiles: one thread per texel (curve c, row j, column i; i
// fastest), so a warp writes neighbouring texels of one or two tiles.  Each
// texel is F(i/s, j/s) of its curve's tile function (see SEIL2S above); the
// unorm range of a tile is that of its four corners (a bilinear function
// takes its extremes there), recorded by the thread of texel (0, 0).
__global__ void k_pack_spread(const CurveArgs a, TexArgs ta, cudaSurfaceObject_t surf, int fmt)
{
    const int sp = ta.sp, n1 = sp + 1;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t c = idx / (n1 * n1);
    if (c >= a.n_curves) return;
    const int r = (int)(idx - c * n1 * n1);
    const int j = r / n1, i = r - j * n1;
    const int d = a.degree, dim = a.dim;
    float4 b[4];
    for (int q = 0; q < 4; ++q) {
        const int pi = q == 0 ? 0 : q == 1 ? 1 : q == 2 ? d - 1 : d;  // b0, b1, b_(d-1), bd
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < dim; ++k) v[k] = load_elem(a.ctrl, a.dtype, (c * (d + 1) + pi) * dim + k);
        b[q] = make_float4(v[0], v[1], v[2], v[3]);
    }
    // d1 = d (b1 - b0) - (bd - b0), d_(d-1) = d (b_(d-1) - bd) - (b0 - bd)  (Sec. 3.1)
    const float fd = (float)d;
    const float4 d1 = sub4(scale4(fd, sub4(b[1], b[0])), sub4(b[3], b[0]));
    const float4 dl = sub4(scale4(fd, sub4(b[2], b[3])), sub4(b[0], b[3]));
    const float inv = 1.f / (float)sp;  // sp a power of two: exact
    auto texel = [&](int x, int y) {
        const float ys = 0.25f * inv * (float)y, xs = inv * (float)x;
        const float4 lo = add4(b[0], scale4(ys, d1)), hi = add4(b[3], scale4(ys, dl));
        return add4(scale4(1.f - xs, lo), scale4(xs, hi));
    };
    const float4 v = texel(i, j);
    const int x0 = (int)(c % ta.tw) * ta.wt, y0 = (int)(c / ta.tw) * ta.ht;
    if (fmt < 2) {
        put(surf, fmt, x0 + i, y0 + j, 0, false, v);
        return;
    }
    const float4 c00 = texel(0, 0), c10 = texel(sp, 0), c01 = texel(0, sp), c11 = texel(sp, sp);
    const float4 lo = min4(min4(c00, c10), min4(c01, c11)), hi = max4(max4(c00, c10), max4(c01, c11));
    float4 sc = sub4(hi, lo);
    sc = make_float4(sc.x > 0.f ? sc.x : 1.f, sc.y > 0.f ? sc.y : 1.f, sc.z > 0.f ? sc.z : 1.f, sc.w > 0.f ? sc.w : 1.f);
    if (i == 0 && j == 0) {
        ta.rescale[2 * c] = lo;
        ta.rescale[2 * c + 1] = sc;
    }
    const float4 u = make_float4(__fdiv_rn(v.x - lo.x, sc.x), __fdiv_rn(v.y - lo.y, sc.y), __fdiv_rn(v.z - lo.z, sc.z),
                                 __fdiv_rn(v.w - lo.w, sc.w));
    put(surf, fmt, x0 + i, y0 + j, 0, false, u);
}

// ---------------------------------------------------------------- evaluators

__device__ __forceinline__ float4 lerp4(float4 a, float4 b, float t)
{
    return make_float4(lerp(a.x, b.x, t), lerp(a.y, b.y, t), lerp(a.z, b.z, t), lerp(a.w, b.w, t));
}

template <int KIND>
__device__ __forceinline__ float4 tex_point(const TexArgs& ta, float xb, float yb, float t)
{
    if (KIND == TK_DC3) return tex3D<float4>(ta.tex, xb + t, yb + t, 0.5f + t);
    if (KIND == TK_HYB3) {
        const float y = yb + t;
        const float4 q0 = tex2D<float4>(ta.tex, xb + t, y);
        const float4 q1 = tex2D<float4>(ta.tex, (xb + 1.f) + t, y);
        return lerp4(q0, q1, t);
    }
    if (KIND == TK_SEIL2) {
        const float st = fmaf(-t, t, t);
        return tex2D<float4>(ta.tex, xb + t, yb + st);
    }
    if (KIND == TK_SEIL2S) {
        const float st = fmaf(-t, t, t);
        const float s = (float)ta.sp;
        return tex2D<float4>(ta.tex, xb + s * t, yb + (4.f * s) * st);
    }
    if (KIND == TK_SEIL3) {
        const float st = fmaf(-t, t, t);
        return tex3D<float4>(ta.tex, xb + t, yb + st, 0.5f + st);
    }
    if (KIND == TK_SEIL3Q) {
        const float st = fmaf(-t, t, t);
        return tex3D<float4>(ta.tex, xb + t, yb + 4.f * st, 0.5f + 16.f * (st * st));
    }
    const int d = ta.deg;
    if (KIND == TK_DCN) {
        if (d == 1) return tex3D<float4>(ta.tex, xb + t, yb, 0.5f);
        if (d == 2) return tex3D<float4>(ta.tex, xb + t, yb + t, 0.5f);
        float4 q[kMaxDegree - 2];
        const float y = yb + t, z = 0.5f + t;
        for (int i = 0; i <= d - 3; ++i) q[i] = tex3D<float4>(ta.tex, (xb + (float)i) + t, y, z);
        for (int r = 1; r <= d - 3; ++r)
            for (int i = 0; i <= d - 3 - r; ++i) q[i] = lerp4(q[i], q[i + 1], t);
        return q[0];
    }
    // TK_HYBN
    if (d == 1) return tex2D<float4>(ta.tex, xb + t, yb);
    float4 q[kMaxDegree - 1];
    const float y = yb + t;
    for (int i = 0; i <= d - 2; ++i) q[i] = tex2D<float4>(ta.tex, (xb + (float)i) + t, y);
    for (int r = 1; r <= d - 2; ++r)
        for (int i = 0; i <= d - 2 - r; ++i) q[i] = lerp4(q[i], q[i + 1], t);
    return q[0];
}

__device__ __forceinline__ float seg_len4(float4 p, float4 q)
{
    const float ex = p.x - q.x, ey = p.y - q.y, ez = p.z - q.z, ew = p.w - q.w;
    return sqrt_approx(fmaf(ew, ew, fmaf(ez, ez, fmaf(ey, ey, ex * ex))));
}

// per-curve (offset, scale) of a unorm tile; identity for float / half texels
struct Rescale {
    float4 lo, sc;
    bool on;
    __device__ __forceinline__ Rescale(const TexArgs& ta, int64_t c) : on(ta.rescale != nullptr)
    {
        if (on) {
            lo = ta.rescale[2 * c];
            sc = ta.rescale[2 * c + 1];
        }
    }
    __device__ __forceinline__ float4 operator()(float4 f) const
    {
        if (!on) return f;
        return make_float4(fmaf(sc.x, f.x, lo.x), fmaf(sc.y, f.y, lo.y), fmaf(sc.z, f.z, lo.z), fmaf(sc.w, f.w, lo.w));
    }
};

template <int KIND, int TM>
__device__ __forceinline__ float4 tex_eval(const CurveArgs& a, const TexArgs& ta, int64_t c, int j, uint32_t kc,
                                           float xb, float yb, const Rescale& rs)
{
    const float t = param<TM>(a, c, j, kc);
    float4 P = rs(tex_point<KIND>(ta, xb, yb, t));
    if (TM == TM_ARRAY && t != t) P = make_float4(t, t, t, t);  // NaN parameter -> NaN point
    return P;
}

template <int KIND, int TM, int OM>
__global__ void __launch_bounds__(kWarps * 32) k_tex(const CurveArgs a, const TexArgs ta)
{
    __shared__ float s_stage[OM == OM_POINTS ? kWarps * 32 * 4 : 1];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t n_warps = (int64_t)gridDim.x * kWarps;
    const int dim = a.dim;
    for (int64_t c = (int64_t)blockIdx.x * kWarps + wib; c < a.n_curves; c += n_warps) {
        const float xb = (float)((int)(c % ta.tw) * ta.wt) + 0.5f;
        const float yb = (float)((int)(c / ta.tw) * ta.ht) + 0.5f;
        const uint32_t kc = (TM == TM_HASH) ? lowbias32(a.key ^ (uint32_t)c) : 0u;
        const Rescale rs(ta, c);
        const int n_t = a.n_t;
        if (OM == OM_POINTS) {
            float* stage = s_stage + wib * 32 * 4;
            for (int j0 = 0; j0 < n_t; j0 += 32) {
                const int j = j0 + lane;
                float4 P = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j < n_t) P = tex_eval<KIND, TM>(a, ta, c, j, kc, xb, yb, rs);
                const float pv[4] = {P.x, P.y, P.z, P.w};
                for (int k = 0; k < dim; ++k) stage[lane * dim + k] = pv[k];
                __syncwarp();
                const int valid = min(32, n_t - j0) * dim;
                float* o = a.out + (c * n_t + j0) * dim;
                for (int idx = lane; idx < valid; idx += 32) o[idx] = stage[idx];
                __syncwarp();
            }
        } else {
            const int chunk = (n_t + 31) / 32;
            const int jb = lane * chunk;
            const int je = min(jb + chunk, n_t);
            float acc = 0.f;
            float4 first = make_float4(0.f, 0.f, 0.f, 0.f), prev = first;
            if (jb < je) {
                first = prev = tex_eval<KIND, TM>(a, ta, c, jb, kc, xb, yb, rs);
#pragma unroll 4
                for (int j = jb + 1; j < je; ++j) {
                    const float4 P = tex_eval<KIND, TM>(a, ta, c, j, kc, xb, yb, rs);
                    acc += seg_len4(P, prev);
                    prev = P;
                }
            }
            float4 pl;
            pl.x = __shfl_up_sync(kFull, prev.x, 1);
            pl.y = __shfl_up_sync(kFull, prev.y, 1);
            pl.z = __shfl_up_sync(kFull, prev.z, 1);
            pl.w = __shfl_up_sync(kFull, prev.w, 1);
            if (lane > 0 && jb < je) acc += seg_len4(first, pl);
            acc = warp_sum(acc);
            if (lane == 0) a.out[c] = acc;
        }
    }
}

// ---------------------------------------------------------------- dispatch

template <int KIND>
LaunchResult launch_kind(const CurveArgs& a, int tm, int om, Atlas& at, int tw, int wt, int ht, int sp, float4* rescale,
                         cudaStream_t s, const LaunchHooks& h)
{
    TexArgs ta{at.tex, tw, wt, a.degree, rescale, ht, sp};
    h.count(h.self);
    if constexpr (KIND == TK_SEIL2S) {
        const int64_t n_texels = a.n_curves * (int64_t)(sp + 1) * (sp + 1);
        k_pack_spread<<<(unsigned)((n_texels + 255) / 256), 256, 0, s>>>(a, ta, at.surf, at.fmt);
    } else {
        k_pack<KIND><<<(unsigned)((a.n_curves + 255) / 256), 256, 0, s>>>(a, ta, at.surf, at.fmt);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return {1, err};
    const void* kern;
    auto pick = [&](auto k) { kern = (const void*)k; };
    if (om == OM_POINTS) {
        if (tm == TM_ARRAY) pick(k_tex<KIND, TM_ARRAY, OM_POINTS>);
        else if (tm == TM_UNIFORM) pick(k_tex<KIND, TM_UNIFORM, OM_POINTS>);
        else pick(k_tex<KIND, TM_HASH, OM_POINTS>);
    } else {
        if (tm == TM_ARRAY) pick(k_tex<KIND, TM_ARRAY, OM_LENGTH>);
        else if (tm == TM_UNIFORM) pick(k_tex<KIND, TM_UNIFORM, OM_LENGTH>);
        else pick(k_tex<KIND, TM_HASH, OM_LENGTH>);
    }
    const int grid = persistent_grid(kern, kWarps * 32, 0, h.sm_count, (a.n_curves + kWarps - 1) / kWarps);
    void* args[] = {(void*)&a, (void*)&ta};
    h.count(h.self);
    h.begin(h.self, s);
    err = cudaLaunchKernel(kern, dim3(grid), dim3(kWarps * 32), args, 0, s);
    h.end(h.self, s);
    return {2, err};
}

// Tiles per atlas row: a power of two near sqrt(n * ht / wt) so that the
// atlas of wt x ht tiles is roughly square (small coordinates keep more
// fractional bits).
static int tiles_per_row(int64_t n, int wt, int max_w, int ht = 2)
{
    int tw = 1;
    while ((int64_t)tw * tw * wt < n * ht && tw * 2 * wt <= max_w) tw *= 2;
    return tw;
}

// texel format of a call: float4 / half4 by the control-point type, or the
// requested unorm format
int texel_format(int dtype, int tex_format)
{
    return tex_format == 1 ? TEXEL_UNORM16 : tex_format == 2 ? TEXEL_UNORM8 : (dtype == 1 ? TEXEL_F16 : TEXEL_F32);
}

// per-tile rescale pairs (lo, scale) of unorm atlases (context scratch, grown on demand)
cudaError_t rescale_buffer(TexState& ts, int fmt, int64_t n, float4** out)
{
    *out = nullptr;
    if (fmt < 2) return cudaSuccess;
    if (ts.rescale_cap < n) {
        if (ts.rescale) {
            cudaError_t e = cudaDeviceSynchronize();  // the old buffer may still be read
            if (e != cudaSuccess) return e;
            cudaFree(ts.rescale);
            ts.rescale = nullptr;
            ts.rescale_cap = 0;
        }
        cudaError_t e = cudaMalloc(&ts.rescale, (size_t)n * 2 * sizeof(float4));
        if (e != cudaSuccess) return e;
        ts.rescale_cap = n;
    }
    *out = ts.rescale;
    return cudaSuccess;
}

LaunchResult launch_tex_curve(const CurveArgs& a, int variant, int tm, int om, int tex_format, int spread,
                              TexState& ts, cudaStream_t s, const LaunchHooks& h)
{
    const int d = a.degree;
    const int fmt = texel_format(a.dtype, tex_format);
    int kind, wt, ht = 2;
    bool is3d;
    if (variant == 6) {  // BEZ_VAR_TEX_DECASTELJAU
        kind = d == 3 ? TK_DC3 : TK_DCN;
        wt = d >= 3 ? d - 1 : 2;
        is3d = true;
    } else if (variant == 8) {  // BEZ_VAR_TEX_HYBRID
        kind = d == 3 ? TK_HYB3 : TK_HYBN;
        wt = d >= 2 ? d : 2;
        is3d = false;
    } else if (spread > 1) {  // BEZ_VAR_TEX_SEILER, degree 2 or 3, spread tile
        kind = TK_SEIL2S;
        wt = ht = spread + 1;
        is3d = false;
    } else {  // BEZ_VAR_TEX_SEILER
        kind = d <= 3 ? TK_SEIL2 : d <= 5 ? TK_SEIL3 : TK_SEIL3Q;
        wt = 2;
        is3d = d > 3;
    }
    const int max_w = is3d ? ts.max3d : ts.max2d_w;
    const int tw = tiles_per_row(a.n_curves, wt, max_w, ht);
    const int64_t rows = (a.n_curves + tw - 1) / tw;
    const int64_t h_needed = rows * ht;
    if (h_needed > (is3d ? ts.max3d : ts.max2d_h)) return {0, cudaErrorInvalidValue};
    Atlas& at = kind == TK_DC3 || kind == TK_DCN ? ts.dc3
                : kind == TK_HYB3 || kind == TK_HYBN ? ts.strip2
                : kind == TK_SEIL2 ? ts.seil2
                : kind == TK_SEIL2S ? ts.seil2s : ts.seil3;   // SEIL3 and SEIL3Q share the 2x2x2 atlas
    cudaError_t e = atlas_ensure(at, tw * wt, (int)h_needed, is3d ? 2 : 0, fmt);
    if (e != cudaSuccess) return {0, e};
    float4* rs = nullptr;
    if ((e = rescale_buffer(ts, fmt, a.n_curves, &rs)) != cudaSuccess) return {0, e};
    const int sp = spread > 1 ? spread : 1;
    switch (kind) {
    case TK_DC3: return launch_kind<TK_DC3>(a, tm, om, at, tw, wt, ht, sp, rs, s, h);
    case TK_DCN: return launch_kind<TK_DCN>(a, tm, om, at, tw, wt, ht, sp, rs, s, h);
    case TK_HYB3: return launch_kind<TK_HYB3>(a, tm, om, at, tw, wt, ht, sp, rs, s, h);
    case TK_HYBN: return launch_kind<TK_HYBN>(a, tm, om, at, tw, wt, ht, sp, rs, s, h);
    case TK_SEIL2: return launch_kind<TK_SEIL2>(a, tm, om, at, tw, wt, ht, sp, rs, s, h);
    case TK_SEIL2S: return launch_kind<TK_SEIL2S>(a, tm, om, at, tw, wt, ht, sp, rs, s, h);
    case TK_SEIL3: return launch_kind<TK_SEIL3>(a, tm, om, at, tw, wt, ht, sp, rs, s, h);
    default: return launch_kind<TK_SEIL3Q>(a, tm, om, at, tw, wt, ht, sp, rs, s, h);
    }
}

// ---------------------------------------------------------------- co-issue

// Sec. 5: a texture evaluator only helps when its reads overlap arithmetic
// that the FP32 pipes would do anyway.  k_coissue evaluates cubic 3D curves
// to polyline lengths with both units in one instruction stream: in every
// group of 8 samples of a lane's run the first S come from the curve's tex2D
// Seiler tile (one bilinear read each, issued first), the other 8 - S from
// centred Horner in registers while those reads are in flight.  Draws are
// those of bez_eval's hash (pre-mixed key, sample indices < 2^16).
template <int S, bool FIRST, bool FULL>
__device__ __forceinline__ void coissue_group(const Eval<VAR_HORNER_CENTRED, 3, 3>& e, const TexArgs& ta, float xb,
                                              float yb, uint32_t kg, int n, float (&first)[3], float (&last)[3],
                                              float& acc, const Rescale& rs)
{
    float4 T[S];
#pragma unroll
    for (int i = 0; i < S; ++i) {
        if (FULL || i < n) {
            const float t = hash_one_plus(lowbias32_premixed(kg ^ (uint32_t)i, 0u)) - 1.0f;
            T[i] = rs(tex2D<float4>(ta.tex, xb + t, yb + fmaf(-t, t, t)));
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (FULL || i < n) {
            float P[3];
            if (i < S) {
                P[0] = T[i < S ? i : 0].x;
                P[1] = T[i < S ? i : 0].y;
                P[2] = T[i < S ? i : 0].z;
            } else {
                DrawEval<Eval<VAR_HORNER_CENTRED, 3, 3>>::at(e, (kg ^ (uint32_t)i) * kLowbiasMul1, P);
            }
            if (FIRST && i == 0) {
#pragma unroll
                for (int k = 0; k < 3; ++k) first[k] = last[k] = P[k];
            } else {
                acc += seg_len<3>(P, last);
#pragma unroll
                for (int k = 0; k < 3; ++k) last[k] = P[k];
            }
        }
    }
}

template <int S>
__global__ void __launch_bounds__(kWarps * 32, S <= 1 ? 5 : 4) k_coissue(const CurveArgs a, const TexArgs ta)
{
    using E = Eval<VAR_HORNER_CENTRED, 3, 3>;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t n_warps = (int64_t)gridDim.x * kWarps;
    int64_t c = (int64_t)blockIdx.x * kWarps + wib;
    CtrlRegs<4, 3> cur;
    cur.load(a, c, 12, lane);
    for (; c < a.n_curves; c += n_warps) {
        float b[4][3];
        cur.unpack(b, 3);
        cur.load(a, c + n_warps, 12, lane);
        E e;
        e.setup(b, 3);
        const uint32_t km = curve_key<TM_HASH16>(a, c);
        const float xb = (float)((int)(c % ta.tw) * ta.wt) + 0.5f;
        const float yb = (float)((int)(c / ta.tw) * 2) + 0.5f;
        const Rescale rs(ta, c);
        const int n_t = a.n_t;
        // 8-aligned runs: sample g + i of a group starting at g has index g ^ i
        const int chunk = ((n_t + 31) / 32 + 7) & ~7;
        const int jb = lane * chunk;
        const int je = min(jb + chunk, n_t);
        float acc = 0.f;
        float first[3] = {0.f, 0.f, 0.f}, last[3] = {0.f, 0.f, 0.f};
        if (jb < je) {
            coissue_group<S, true, false>(e, ta, xb, yb, km ^ (uint32_t)jb, je - jb, first, last, acc, rs);
            int g = jb + 8;
            for (; g + 8 <= je; g += 8)
                coissue_group<S, false, true>(e, ta, xb, yb, km ^ (uint32_t)g, 8, first, last, acc, rs);
            if (g < je) coissue_group<S, false, false>(e, ta, xb, yb, km ^ (uint32_t)g, je - g, first, last, acc, rs);
        }
        float pl[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) pl[k] = __shfl_up_sync(kFull, last[k], 1);
        if (lane > 0 && jb < je) acc += seg_len<3>(first, pl);
        acc = warp_sum(acc);
        if (lane == 0) a.out[c] = acc;
    }
}

LaunchResult launch_tex_coissue(const CurveArgs& a, int share, int tex_format, TexState& ts, cudaStream_t s,
                                const LaunchHooks& h)
{
    const int wt = 2;
    const int tw = tiles_per_row(a.n_curves, wt, ts.max2d_w);
    const int64_t rows = (a.n_curves + tw - 1) / tw;
    if (rows * 2 > ts.max2d_h) return {0, cudaErrorInvalidValue};
    const int fmt = texel_format(a.dtype, tex_format);
    cudaError_t e = atlas_ensure(ts.seil2, tw * wt, (int)(rows * 2), 0, fmt);
    if (e != cudaSuccess) return {0, e};
    float4* rs = nullptr;
    if ((e = rescale_buffer(ts, fmt, a.n_curves, &rs)) != cudaSuccess) return {0, e};
    TexArgs ta{ts.seil2.tex, tw, wt, 3, rs, 2, 1};
    h.count(h.self);
    k_pack<TK_SEIL2><<<(unsigned)((a.n_curves + 255) / 256), 256, 0, s>>>(a, ta, ts.seil2.surf, fmt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return {1, e};
    const void* kern;
    switch (share) {
    case 1: kern = (const void*)k_coissue<1>; break;
    case 2: kern = (const void*)k_coissue<2>; break;
    case 3: kern = (const void*)k_coissue<3>; break;
    case 4: kern = (const void*)k_coissue<4>; break;
    case 5: kern = (const void*)k_coissue<5>; break;
    case 6: kern = (const void*)k_coissue<6>; break;
    default: kern = (const void*)k_coissue<7>; break;
    }
    const int64_t work = (a.n_curves + kWarps - 1) / kWarps;
    int grid = persistent_grid(kern, kWarps * 32, 0, h.sm_count, work);
    if (work > grid) {
        // as for k_curve: blocks of kCurvesPerWarp curves per warp
        const int64_t g = (a.n_curves + (int64_t)kWarps * kCurvesPerWarp - 1) / ((int64_t)kWarps * kCurvesPerWarp);
        if (g > grid) grid = (int)(g < 2147483647 ? g : 2147483647);
    }
    void* args[] = {(void*)&a, (void*)&ta};
    h.count(h.self);
    h.begin(h.self, s);
    e = cudaLaunchKernel(kern, dim3(grid), dim3(kWarps * 32), args, 0, s);
    h.end(h.self, s);
    return {2, e};
}

// ---------------------------------------------------------------- zig-zag C0 chains

// Sec. 2.1 (Eq. 1-2, Fig. 2): N quadratic segments with shared end points in
// an (N+1) x 2 texture.  Column k holds P_(2k) in row k mod 2 and a free
// texel F_k in the other row.  Segment k is read between (k, k mod 2) and
// (k+1, 1 - k mod 2); bilinear filtering there gives
//   (1-tau)^2 P_2k + tau (1-tau) (F_k + F_(k+1)) + tau^2 P_(2k+2),
// the quadratic with middle point (F_k + F_(k+1)) / 2, so the N constraints
// are F_k + F_(k+1) = 2 P_(2k+1) on N+1 unknowns.  The free choice of F_0
// (per component) minimises max_k |F_k|: with F_k = (-1)^k F_0 + G_k,
// F_0 = -(max_k H_k + min_k H_k) / 2 for H_k = (-1)^k G_k.  Each F_(k+1) is
// formed from the stored F_k, so every constraint holds to one rounding.
//
// Reads.  Along segment k both axes take the same fraction (tau on even k,
// 1 - tau on odd k), so the hardware's per-axis weight rounding moves the
// read along the curve: (tau~ - tau) Q'(tau) plus the twist weight's
// rounding times the window's twist P_2k - 2 P_(2k+1) + P_(2k+2).  That holds
// only if both coordinates carry the same fraction bits; the FP32 sums of the
// atlas offsets would round them differently, and a read whose two 8-bit
// weights round in opposite directions is off by 2^-8 of the free texels,
// which can be tens of times the segment size.  The evaluator therefore
// snaps the fraction to the hardware's 1/256 grid itself (round half up, as
// the filter does) and adds it to exact integer coordinates (atlas width and
// height below 2^15, so the sums are exact).
//
// Spread s >= 2: every window's bilinear function is sampled on an
// (s+1) x (s+1) texel grid (neighbouring windows share their boundary
// column, where both functions interpolate the same two texels), the
// texture is (N s + 1) x (s + 1), and segment k is read at
// (s (k + tau), s tau) or (s (k + tau), s (1 - tau)); the rounding terms
// shrink by s (the twist term by s^2).
// free texel F_0 of a quadratic chain: the minimax start (smallest largest
// |F_k| over the chain)
__device__ __forceinline__ float4 chain_f0(const CurveArgs& a, int64_t base)
{
    const int N = a.n_seg, dim = a.dim;
    float f0[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < dim; ++k) {
        float g = 0.f, hmax = 0.f, hmin = 0.f;  // G_0 = 0
        for (int s = 0; s < N; ++s) {
            g = 2.f * load_elem(a.ctrl, a.dtype, base + (int64_t)(2 * s + 1) * dim + k) - g;  // G_(s+1)
            const float h = (s & 1) ? g : -g;   // H_(s+1) = (-1)^(s+1) G_(s+1)
            hmax = fmaxf(hmax, h);
            hmin = fminf(hmin, h);
        }
        f0[k] = -0.5f * (hmax + hmin);
    }
    return make_float4(f0[0], f0[1], f0[2], f0[3]);
}

// Unorm16 chain texels: the chain's per-component range over its column
// texels P_2k and F_k (every spread texel is a convex combination of them),
// recorded as (lo, scale) in rescale[2 c], rescale[2 c + 1].  Texels store
// (v - lo) / scale and the evaluator maps the filtered value back by
// lo + scale * f.
__device__ __forceinline__ void chain_range(const CurveArgs& a, int64_t base, float4 F, float4& lo, float4& sc)
{
    const int N = a.n_seg, dim = a.dim;
    float4 hi = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
    lo = make_float4(INFINITY, INFINITY, INFINITY, INFINITY);
    for (int s = 0; s <= N; ++s) {
        float p[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < dim; ++k) p[k] = load_elem(a.ctrl, a.dtype, base + (int64_t)(2 * s) * dim + k);
        const float4 Pe = make_float4(p[0], p[1], p[2], p[3]);
        lo = min4(lo, min4(Pe, F));
        hi = max4(hi, max4(Pe, F));
        if (s < N) {
            float m[4] = {0.f, 0.f, 0.f, 0.f};
            for (int k = 0; k < dim; ++k) m[k] = load_elem(a.ctrl, a.dtype, base + (int64_t)(2 * s + 1) * dim + k);
            F = make_float4(2.f * m[0] - F.x, 2.f * m[1] - F.y, 2.f * m[2] - F.z, 2.f * m[3] - F.w);
        }
    }
    sc = sub4(hi, lo);
    sc = make_float4(sc.x > 0.f ? sc.x : 1.f, sc.y > 0.f ? sc.y : 1.f, sc.z > 0.f ? sc.z : 1.f, sc.w > 0.f ? sc.w : 1.f);
}

__device__ __forceinline__ float4 unorm_of(float4 v, float4 lo, float4 sc)
{
    return make_float4(__fdiv_rn(v.x - lo.x, sc.x), __fdiv_rn(v.y - lo.y, sc.y), __fdiv_rn(v.z - lo.z, sc.z),
                       __fdiv_rn(v.w - lo.w, sc.w));
}

__global__ void k_chain_pack(const CurveArgs a, int cw, cudaSurfaceObject_t surf, int fmt, float4* rescale)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.n_curves) return;
    const int N = a.n_seg, dim = a.dim;
    const int64_t base = c * (int64_t)(2 * N + 1) * dim;
    auto P = [&](int i, int k) { return load_elem(a.ctrl, a.dtype, base + (int64_t)i * dim + k); };
    const int x0 = (int)(c % cw) * (N + 1), y0 = (int)(c / cw) * 2;
    float4 F = chain_f0(a, base);
    const bool un = fmt == TEXEL_UNORM16;
    float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), sc = make_float4(1.f, 1.f, 1.f, 1.f);
    if (un) {
        chain_range(a, base, F, lo, sc);
        rescale[2 * c] = lo;
        rescale[2 * c + 1] = sc;
    }
    for (int s = 0; s <= N; ++s) {
        float p[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < dim; ++k) p[k] = P(2 * s, k);
        const float4 Pe = make_float4(p[0], p[1], p[2], p[3]);
        const bool hw = fmt == 1;
        if (hw) {  // store what the half texture holds, so the next constraint uses it
            F = make_float4(__half2float(__float2half_rn(F.x)), __half2float(__float2half_rn(F.y)),
                            __half2float(__float2half_rn(F.z)), __half2float(__float2half_rn(F.w)));
        }
        put(surf, fmt, x0 + s, y0 + (s & 1), 0, false, un ? unorm_of(Pe, lo, sc) : Pe);
        put(surf, fmt, x0 + s, y0 + 1 - (s & 1), 0, false, un ? unorm_of(F, lo, sc) : F);
        if (s < N) {
            float m[4] = {0.f, 0.f, 0.f, 0.f};
            for (int k = 0; k < dim; ++k) m[k] = P(2 * s + 1, k);
            F = make_float4(2.f * m[0] - F.x, 2.f * m[1] - F.y, 2.f * m[2] - F.z, 2.f * m[3] - F.w);
        }
    }
}

// Spread chain texture: one warp per chain.  Lane 0 solves the free texels
// F_k as k_chain_pack does and stages the column texels (P_2k, F_k) in shared
// memory; then the lanes write the (N s + 1) x (s + 1) grid column by column.
constexpr int kChainPackWarps = 4;
constexpr size_t kChainPackMaxSmem = 192 * 1024;  // spread chains up to 1534 segments
__global__ void __launch_bounds__(kChainPackWarps * 32) k_chain_pack_spread(const CurveArgs a, int cw, int sp,
                                                                            cudaSurfaceObject_t surf, int fmt,
                                                                            float4* rescale)
{
    extern __shared__ float4 s_cols[];  // per warp: [N+1] P_2k, then [N+1] F_k, then (lo, scale)
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * kChainPackWarps + wib;
    if (c >= a.n_curves) return;
    const int N = a.n_seg, dim = a.dim;
    float4* Pc = s_cols + (size_t)wib * (2 * (N + 1) + 2);
    float4* Fc = Pc + (N + 1);
    float4* Rs = Fc + (N + 1);
    const int64_t base = c * (int64_t)(2 * N + 1) * dim;
    auto P = [&](int i, int k) { return load_elem(a.ctrl, a.dtype, base + (int64_t)i * dim + k); };
    const bool un = fmt == TEXEL_UNORM16;
    if (lane == 0) {
        float4 F = chain_f0(a, base);
        if (un) {
            float4 lo, sc;
            chain_range(a, base, F, lo, sc);
            rescale[2 * c] = Rs[0] = lo;
            rescale[2 * c + 1] = Rs[1] = sc;
        }
        for (int s = 0; s <= N; ++s) {
            float p[4] = {0.f, 0.f, 0.f, 0.f};
            for (int k = 0; k < dim; ++k) p[k] = P(2 * s, k);
            if (fmt == 1)
                F = make_float4(__half2float(__float2half_rn(F.x)), __half2float(__float2half_rn(F.y)),
                                __half2float(__float2half_rn(F.z)), __half2float(__float2half_rn(F.w)));
            Pc[s] = make_float4(p[0], p[1], p[2], p[3]);
            Fc[s] = F;
            if (s < N) {
                float m[4] = {0.f, 0.f, 0.f, 0.f};
                for (int k = 0; k < dim; ++k) m[k] = P(2 * s + 1, k);
                F = make_float4(2.f * m[0] - F.x, 2.f * m[1] - F.y, 2.f * m[2] - F.z, 2.f * m[3] - F.w);
            }
        }
    }
    __syncwarp();
    const int W = N * sp + 1;
    const int x0 = (int)(c % cw) * W, y0 = (int)(c / cw) * (sp + 1);
    const float inv = 1.f / (float)sp;  // sp a power of two: exact
    for (int i = lane; i < W; i += 32) {
        const int k = min(i / sp, N - 1);
        const float xs = inv * (float)(i - k * sp);
        // window k: row r of column k holds P_2k if r == k mod 2, else F_k
        const int rk = k & 1, rk1 = (k + 1) & 1;
        const float4 t00 = rk == 0 ? Pc[k] : Fc[k], t01 = rk == 0 ? Fc[k] : Pc[k];
        const float4 t10 = rk1 == 0 ? Pc[k + 1] : Fc[k + 1], t11 = rk1 == 0 ? Fc[k + 1] : Pc[k + 1];
        const float4 r0 = add4(scale4(1.f - xs, t00), scale4(xs, t10));
        const float4 r1 = add4(scale4(1.f - xs, t01), scale4(xs, t11));
        for (int j = 0; j <= sp; ++j) {
            const float ys = inv * (float)j;
            const float4 v = add4(scale4(1.f - ys, r0), scale4(ys, r1));
            put(surf, fmt, x0 + i, y0 + j, 0, false, un ? unorm_of(v, Rs[0], Rs[1]) : v);
        }
    }
}

// Cubic C0 chains (Sec. 2.1, last paragraph: two quadratic chains front to
// back in a 3D texture, interpolated to a cubic).  Column k of an
// (N+1) x 2 x 2 texture has its corner at (y, z) = (k mod 2, k mod 2),
// holding P_3k; the texels with y flipped (a_k), z flipped (b_k) and both
// flipped (d_k) are free.  A trilinear read of columns k, k+1 from the
// corner at (tau, tau, tau) weighs a texel by tau^m (1 - tau)^(3-m), m its
// number of flips, so it evaluates the cubic whose control points are the
// means of the texels with m = 0..3: P_3k, (a_k + b_k + d_(k+1)) / 3,
// (d_k + a_(k+1) + b_(k+1)) / 3, P_3k+3 -- the three-texel form of the
// E = (B + C) / 2 identity.  With s_k = a_k + b_k the constraints are
// d_(k+1) = 3 P_(3k+1) - s_k and s_(k+1) = 3 P_(3k+2) - d_k: two
// interleaved chains (s_0, d_1, s_2, ... and d_0, s_1, d_2, ...) with one
// free start each, chosen per component like F_0 above (minimax), and
// a_k = b_k = s_k / 2.  Each z slice is then a quadratic zig-zag chain (the
// slice through a segment's corner reads a quadratic starting at P_3k, the
// other one ending at P_3k+3), and the z weight lerps them.
__global__ void k_chain3_pack(const CurveArgs a, int cw, cudaSurfaceObject_t surf, int fmt)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.n_curves) return;
    const int N = a.n_seg, dim = a.dim;
    const int64_t base = c * (int64_t)(3 * N + 1) * dim;
    auto P = [&](int i, int k) { return load_elem(a.ctrl, a.dtype, base + (int64_t)i * dim + k); };
    // chain A: x_0 = s_0, x_(k+1) = 3 P[k even ? 3k+1 : 3k+2] - x_k;
    // chain B: y_0 = d_0, y_(k+1) = 3 P[k even ? 3k+2 : 3k+1] - y_k
    float xa0[4] = {0.f, 0.f, 0.f, 0.f}, yb0[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < dim; ++k) {
        float ga = 0.f, gb = 0.f, amax = 0.f, amin = 0.f, bmax = 0.f, bmin = 0.f;
        for (int s = 0; s < N; ++s) {
            ga = 3.f * P((s & 1) ? 3 * s + 2 : 3 * s + 1, k) - ga;
            gb = 3.f * P((s & 1) ? 3 * s + 1 : 3 * s + 2, k) - gb;
            const float ha = (s & 1) ? ga : -ga, hb = (s & 1) ? gb : -gb;  // (-1)^(s+1) G_(s+1)
            amax = fmaxf(amax, ha);
            amin = fminf(amin, ha);
            bmax = fmaxf(bmax, hb);
            bmin = fminf(bmin, hb);
        }
        xa0[k] = -0.5f * (amax + amin);
        yb0[k] = -0.5f * (bmax + bmin);
    }
    const int x0 = (int)(c % cw) * (N + 1), y0 = (int)(c / cw) * 2;
    float4 X = make_float4(xa0[0], xa0[1], xa0[2], xa0[3]), Y = make_float4(yb0[0], yb0[1], yb0[2], yb0[3]);
    auto stored = [&](float4 v) {
        if (fmt != 1) return v;  // half texels: continue the recurrence from what the texture holds
        return make_float4(__half2float(__float2half_rn(v.x)), __half2float(__float2half_rn(v.y)),
                           __half2float(__float2half_rn(v.z)), __half2float(__float2half_rn(v.w)));
    };
    for (int s = 0; s <= N; ++s) {
        const int cc = s & 1;
        const float4 sk = (s & 1) ? Y : X, dk = (s & 1) ? X : Y;   // s_k, d_k
        float4 ak = scale4(0.5f, sk);
        ak = stored(ak);
        const float4 bk = stored(sub4(sk, ak)), dks = stored(dk);
        float p[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < dim; ++k) p[k] = P(3 * s, k);
        put(surf, fmt, x0 + s, y0 + cc, cc, true, make_float4(p[0], p[1], p[2], p[3]));
        put(surf, fmt, x0 + s, y0 + 1 - cc, cc, true, ak);
        put(surf, fmt, x0 + s, y0 + cc, 1 - cc, true, bk);
        put(surf, fmt, x0 + s, y0 + 1 - cc, 1 - cc, true, dks);
        if (s < N) {
            // the stored s_k (a_k + b_k) and d_k continue the recurrences
            const float4 ss = add4(ak, bk);
            float m1[4] = {0.f, 0.f, 0.f, 0.f}, m2[4] = {0.f, 0.f, 0.f, 0.f};
            for (int k = 0; k < dim; ++k) {
                m1[k] = P(3 * s + 1, k);
                m2[k] = P(3 * s + 2, k);
            }
            const float4 dn = make_float4(3.f * m1[0] - ss.x, 3.f * m1[1] - ss.y, 3.f * m1[2] - ss.z, 3.f * m1[3] - ss.w);
            const float4 sn = make_float4(3.f * m2[0] - dks.x, 3.f * m2[1] - dks.y, 3.f * m2[2] - dks.z,
                                          3.f * m2[3] - dks.w);
            // next column: s_(k+1) = sn, d_(k+1) = dn; chain A holds s on even, d on odd columns
            if ((s + 1) & 1) {
                X = dn;
                Y = sn;
            } else {
                X = sn;
                Y = dn;
            }
        }
    }
}

template <int TM>
__device__ __forceinline__ float4 zigzag_eval(const CurveArgs& a, cudaTextureObject_t tex, int64_t c, int j,
                                              uint32_t kc, float xb, float yb, int sp, bool cubic = false)
{
    const float ns = (float)a.n_seg;
    float t;
    if (TM == TM_ARRAY) {
        t = __ldg(a.t + c * a.t_stride + j);
        t = t < 0.f ? 0.f : (t > ns ? ns : t);
    } else if (TM == TM_UNIFORM) {
        t = ns * (a.n_t > 1 ? __fdiv_rn((float)j, (float)(a.n_t - 1)) : 0.f);
    } else {
        t = ns * hash_unit(lowbias32(kc ^ (uint32_t)j));
    }
    int k = (int)floorf(t);
    k = k < 0 ? 0 : (k > a.n_seg - 1 ? a.n_seg - 1 : k);
    const float tau = t - (float)k;
    // u = s tau = iu + fq with fq on the filter's 1/256 grid (round half up)
    const float u = (float)sp * tau;
    float iu = floorf(u);
    float fq = floorf(fmaf(u - iu, 256.f, 0.5f)) * (1.f / 256.f);
    if (fq >= 1.f) {
        iu += 1.f;
        fq = 0.f;
    }
    // odd segments run from row s down to row 0: s (1 - tau) = (s - iu - 1) + (1 - fq)
    const bool odd = k & 1;
    const float iy = odd ? (float)sp - iu - (fq > 0.f ? 1.f : 0.f) : iu;
    const float fy = odd ? (fq > 0.f ? 1.f - fq : 0.f) : fq;
    float4 P;
    if (cubic)  // z runs like y: from slice k mod 2 to the other
        P = tex3D<float4>(tex, (xb + ((float)(k * sp) + iu)) + fq, (yb + iy) + fy, (0.5f + iy) + fy);
    else
        P = tex2D<float4>(tex, (xb + ((float)(k * sp) + iu)) + fq, (yb + iy) + fy);
    if (TM == TM_ARRAY && t != t) P = make_float4(t, t, t, t);
    return P;
}

template <int TM, int OM, bool CUBIC = false>
__global__ void __launch_bounds__(kWarps * 32) k_chain_tex(const CurveArgs a, cudaTextureObject_t tex, int cw, int sp,
                                                           const float4* rescale)
{
    __shared__ float s_stage[OM == OM_POINTS ? kWarps * 32 * 4 : 1];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t n_warps = (int64_t)gridDim.x * kWarps;
    const int dim = a.dim;
    for (int64_t c = (int64_t)blockIdx.x * kWarps + wib; c < a.n_curves; c += n_warps) {
        const float xb = (float)((int)(c % cw) * (a.n_seg * sp + 1)) + 0.5f;
        const float yb = (float)((int)(c / cw) * (sp + 1)) + 0.5f;
        const uint32_t kc = (TM == TM_HASH) ? lowbias32(a.key ^ (uint32_t)c) : 0u;
        const int n_t = a.n_t;
        // unorm16 texels: the filtered value maps back by lo + scale * f
        float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), sc = make_float4(1.f, 1.f, 1.f, 1.f);
        if (rescale) {
            lo = rescale[2 * c];
            sc = rescale[2 * c + 1];
        }
        auto point = [&](int j) {
            const float4 f = zigzag_eval<TM>(a, tex, c, j, kc, xb, yb, sp, CUBIC);
            if (!rescale) return f;
            return make_float4(fmaf(sc.x, f.x, lo.x), fmaf(sc.y, f.y, lo.y), fmaf(sc.z, f.z, lo.z),
                               fmaf(sc.w, f.w, lo.w));
        };
        if (OM == OM_POINTS) {
            float* stage = s_stage + wib * 32 * 4;
            for (int j0 = 0; j0 < n_t; j0 += 32) {
                const int j = j0 + lane;
                float4 P = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j < n_t) P = point(j);
                const float pv[4] = {P.x, P.y, P.z, P.w};
                for (int k = 0; k < dim; ++k) stage[lane * dim + k] = pv[k];
                __syncwarp();
                const int valid = min(32, n_t - j0) * dim;
                float* o = a.out + (c * n_t + j0) * dim;
                for (int idx = lane; idx < valid; idx += 32) o[idx] = stage[idx];
                __syncwarp();
            }
        } else {
            const int chunk = (n_t + 31) / 32;
            const int jb = lane * chunk;
            const int je = min(jb + chunk, n_t);
            float acc = 0.f;
            float4 first = make_float4(0.f, 0.f, 0.f, 0.f), prev = first;
            if (jb < je) {
                first = prev = point(jb);
#pragma unroll 4
                for (int j = jb + 1; j < je; ++j) {
                    const float4 P = point(j);
                    acc += seg_len4(P, prev);
                    prev = P;
                }
            }
            float4 pl;
            pl.x = __shfl_up_sync(kFull, prev.x, 1);
            pl.y = __shfl_up_sync(kFull, prev.y, 1);
            pl.z = __shfl_up_sync(kFull, prev.z, 1);
            pl.w = __shfl_up_sync(kFull, prev.w, 1);
            if (lane > 0 && jb < je) acc += seg_len4(first, pl);
            acc = warp_sum(acc);
            if (lane == 0) a.out[c] = acc;
        }
    }
}

// Chain atlases stay below 2^15 texels per axis so that the snapped read
// coordinates (integer + 8-bit fraction) are exact in FP32.
constexpr int kChainMaxCoord = 32768;

// Cubic chains: (N+1) x 2 x 2 texels per chain in a 3D atlas of depth 2.
static LaunchResult launch_tex_chain3(const CurveArgs& a, int tm, int om, TexState& ts, cudaStream_t s,
                                     const LaunchHooks& h)
{
    const int64_t wt64 = (int64_t)a.n_seg + 1;
    const int max_w = ts.max3d < kChainMaxCoord ? ts.max3d : kChainMaxCoord;
    if (wt64 > max_w) return {0, cudaErrorInvalidValue};
    const int wt = (int)wt64;
    const int fmt = a.dtype == 1 ? 1 : 0;
    const int cw = tiles_per_row(a.n_curves, wt, max_w, 2);
    const int64_t h_needed = (a.n_curves + cw - 1) / cw * 2;
    if (h_needed > max_w || (int64_t)cw * wt > max_w) return {0, cudaErrorInvalidValue};
    cudaError_t e = atlas_ensure(ts.chain3, cw * wt, (int)h_needed, 2, fmt);
    if (e != cudaSuccess) return {0, e};
    h.count(h.self);
    k_chain3_pack<<<(unsigned)((a.n_curves + 127) / 128), 128, 0, s>>>(a, cw, ts.chain3.surf, fmt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return {1, e};
    const void* kern;
    if (om == OM_POINTS)
        kern = tm == TM_ARRAY ? (const void*)k_chain_tex<TM_ARRAY, OM_POINTS, true>
               : tm == TM_UNIFORM ? (const void*)k_chain_tex<TM_UNIFORM, OM_POINTS, true>
                                  : (const void*)k_chain_tex<TM_HASH, OM_POINTS, true>;
    else
        kern = tm == TM_ARRAY ? (const void*)k_chain_tex<TM_ARRAY, OM_LENGTH, true>
               : tm == TM_UNIFORM ? (const void*)k_chain_tex<TM_UNIFORM, OM_LENGTH, true>
                                  : (const void*)k_chain_tex<TM_HASH, OM_LENGTH, true>;
    const int grid = persistent_grid(kern, kWarps * 32, 0, h.sm_count, (a.n_curves + kWarps - 1) / kWarps);
    cudaTextureObject_t tex = ts.chain3.tex;
    int cw_arg = cw, sp_arg = 1;
    const float4* no_rescale = nullptr;
    void* args[] = {(void*)&a, (void*)&tex, (void*)&cw_arg, (void*)&sp_arg, (void*)&no_rescale};
    h.count(h.self);
    h.begin(h.self, s);
    e = cudaLaunchKernel(kern, dim3(grid), dim3(kWarps * 32), args, 0, s);
    h.end(h.self, s);
    return {2, e};
}

LaunchResult launch_tex_chain(const CurveArgs& a, int tm, int om, int spread, int tex_format, TexState& ts,
                              cudaStream_t s, const LaunchHooks& h)
{
    if (a.degree == 3) return launch_tex_chain3(a, tm, om, ts, s, h);
    const int sp = spread > 1 ? spread : 1;
    const int64_t wt64 = (int64_t)a.n_seg * sp + 1;
    const int max_w = ts.max2d_w < kChainMaxCoord ? ts.max2d_w : kChainMaxCoord;
    const int max_h = ts.max2d_h < kChainMaxCoord ? ts.max2d_h : kChainMaxCoord;
    if (wt64 > max_w) return {0, cudaErrorInvalidValue};
    const int wt = (int)wt64;
    const int fmt = tex_format == BEZ_TEX_UNORM16 ? TEXEL_UNORM16 : a.dtype == 1 ? TEXEL_F16 : TEXEL_F32;
    const int cw = tiles_per_row(a.n_curves, wt, max_w, sp + 1);
    const int64_t h_needed = (a.n_curves + cw - 1) / cw * (sp + 1);
    if (h_needed > max_h || (int64_t)cw * wt > max_w) return {0, cudaErrorInvalidValue};
    cudaError_t e = atlas_ensure(ts.chain, cw * wt, (int)h_needed, 0, fmt);
    if (e != cudaSuccess) return {0, e};
    float4* rs = nullptr;
    if ((e = rescale_buffer(ts, fmt, a.n_curves, &rs)) != cudaSuccess) return {0, e};
    h.count(h.self);
    if (sp == 1) {
        k_chain_pack<<<(unsigned)((a.n_curves + 127) / 128), 128, 0, s>>>(a, cw, ts.chain.surf, fmt, rs);
    } else {
        const size_t smem = (size_t)kChainPackWarps * (2 * (a.n_seg + 1) + 2) * sizeof(float4);
        if (smem > kChainPackMaxSmem) return {0, cudaErrorInvalidValue};
        if (smem > 48 * 1024) {
            e = cudaFuncSetAttribute(k_chain_pack_spread, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return {0, e};
        }
        k_chain_pack_spread<<<(unsigned)((a.n_curves + kChainPackWarps - 1) / kChainPackWarps), kChainPackWarps * 32,
                              smem, s>>>(a, cw, sp, ts.chain.surf, fmt, rs);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return {1, e};
    const void* kern;
    if (om == OM_POINTS)
        kern = tm == TM_ARRAY ? (const void*)k_chain_tex<TM_ARRAY, OM_POINTS>
               : tm == TM_UNIFORM ? (const void*)k_chain_tex<TM_UNIFORM, OM_POINTS>
                                  : (const void*)k_chain_tex<TM_HASH, OM_POINTS>;
    else
        kern = tm == TM_ARRAY ? (const void*)k_chain_tex<TM_ARRAY, OM_LENGTH>
               : tm == TM_UNIFORM ? (const void*)k_chain_tex<TM_UNIFORM, OM_LENGTH>
                                  : (const void*)k_chain_tex<TM_HASH, OM_LENGTH>;
    const int grid = persistent_grid(kern, kWarps * 32, 0, h.sm_count, (a.n_curves + kWarps - 1) / kWarps);
    cudaTextureObject_t tex = ts.chain.tex;
    int cw_arg = cw, sp_arg = sp;
    const float4* rs_arg = rs;
    void* args[] = {(void*)&a, (void*)&tex, (void*)&cw_arg, (void*)&sp_arg, (void*)&rs_arg};
    h.count(h.self);
    h.begin(h.self, s);
    e = cudaLaunchKernel(kern, dim3(grid), dim3(kWarps * 32), args, 0, s);
    h.end(h.self, s);
    return {2, e};
}

// ---------------------------------------------------------------- weight probe

__global__ void k_probe_pack(cudaSurfaceObject_t surf)
{
    const int x = threadIdx.x & 1, y = (threadIdx.x >> 1) & 1, z = threadIdx.x >> 2;
    surf3Dwrite(make_float4((float)x, (float)y, (float)z, 1.f), surf, x * 16, y, z);
}

__global__ void k_probe(cudaTextureObject_t tex, const float* xyz, int64_t n, float* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 v = tex3D<float4>(tex, xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]);
    reinterpret_cast<float4*>(out)[i] = v;
}

LaunchResult launch_tex_probe(const float* xyz, int64_t n, float* out, TexState& ts, cudaStream_t s,
                              const LaunchHooks& h)
{
    cudaError_t e = atlas_ensure(ts.probe, 2, 2, 2, 0);
    if (e != cudaSuccess) return {0, e};
    h.count(h.self);
    k_probe_pack<<<1, 8, 0, s>>>(ts.probe.surf);
    e = cudaGetLastError();
    if (e != cudaSuccess || n == 0) return {1, e};
    h.count(h.self);
    h.begin(h.self, s);
    k_probe<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ts.probe.tex, xyz, n, out);
    e = cudaGetLastError();
    h.end(h.self, s);
    return {2, e};
}

// 2D probe: texel (x, y) of a 2x2 float4 texture holds the unit vector of
// channel x + 2 y, so a bilinear read returns the four texel weights.
__global__ void k_probe2_pack(cudaSurfaceObject_t surf)
{
    const int x = threadIdx.x & 1, y = threadIdx.x >> 1;
    const int k = x + 2 * y;
    surf2Dwrite(make_float4(k == 0 ? 1.f : 0.f, k == 1 ? 1.f : 0.f, k == 2 ? 1.f : 0.f, k == 3 ? 1.f : 0.f), surf,
                x * 16, y);
}

__global__ void k_probe2(cudaTextureObject_t tex, const float* xy, int64_t n, float* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    reinterpret_cast<float4*>(out)[i] = tex2D<float4>(tex, xy[2 * i], xy[2 * i + 1]);
}

LaunchResult launch_tex_probe2d(const float* xy, int64_t n, float* out, TexState& ts, cudaStream_t s,
                                const LaunchHooks& h)
{
    cudaError_t e = atlas_ensure(ts.probe2, 2, 2, 0, 0);
    if (e != cudaSuccess) return {0, e};
    h.count(h.self);
    k_probe2_pack<<<1, 4, 0, s>>>(ts.probe2.surf);
    e = cudaGetLastError();
    if (e != cudaSuccess || n == 0) return {1, e};
    h.count(h.self);
    k_probe2<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ts.probe2.tex, xy, n, out);
    return {2, cudaGetLastError()};
}

}  // namespace bez
