// tensor.cu -- tensor-product Bezier surfaces and volumes on uniform grids
// (paper Sec. 2.2: a surface splits its order between u and v, a volume
// between u, v and w; the bicubic case evaluates the four column curves at u
// and then the isoline cubic in v).
//
// Separable contraction, one block per patch (grid-stride; bicubic 3D
// patches on grids of up to 64 rows take one warp per patch, and tricubic
// scalar volumes one warp per volume: k_volume_tricubic1_warp in
// tensor_common.cuh, shared with the texture volumes):
//   surface  X[a][j] = sum_i Bu[a][i] C[i][j]          (isoline control points)
//            P[a][b] = sum_j X[a][j] Bv[b][j]
//   volume   Y[a][j][l] = sum_i Bu[a][i] C[i][j][l]
//            Z[a][b][l] = sum_j Bv[b][j] Y[a][j][l]
//            V[a][b][c] = sum_l Bw[c][l] Z[a][b][l]
// with Bernstein tables of the grid values t_a = fl32(a) / fl32(n-1) built
// once per block.  The output is write-bound; every thread writes runs of
// consecutive floats (float4 when the layout allows), so stores are fully
// coalesced.  The contraction has a reduction depth of 4 for bicubic
// patches, far too small to keep tensor cores busy on a store-bound kernel,
// so it runs on the FP32 pipes.
#include "tensor_common.cuh"

namespace bez {

// Fast path: bicubic 3D patches, nv a multiple of 4.  Each thread owns four
// consecutive points of one grid row and writes them as three float4.
__global__ void __launch_bounds__(kTensorThreads) k_surface_bicubic3(const TensorArgs a)
{
    __shared__ float4 s_bv[kTensorMaxGrid];        // Bv[b][0..3]
    __shared__ float s_bu[kTensorMaxGrid * 4];     // Bu[a][0..3]
    __shared__ float s_c[48];                      // C[i][j][k]
    __shared__ float s_x[kTensorMaxGrid * 12];     // X[a][j][k]
    const int tid = threadIdx.x;
    bernstein_table(s_bu, a.nu, 3, tid, kTensorThreads);
    {
        float* bv = reinterpret_cast<float*>(s_bv);
        bernstein_table(bv, a.nv, 3, tid, kTensorThreads);
    }
    const int nu = a.nu, nv = a.nv;
    const int quads_per_row = nv / 4;
    const int n_quads = nu * quads_per_row;
    const int64_t pts = (int64_t)nu * nv;
    // the next patch's control points are loaded while the current one is
    // evaluated and stored
    float nxt = (tid < 48 && (int64_t)blockIdx.x < a.n) ? load_elem(a.ctrl, a.dtype, (int64_t)blockIdx.x * 48 + tid) : 0.f;
    for (int64_t p = blockIdx.x; p < a.n; p += gridDim.x) {
        __syncthreads();  // tables ready / previous patch done with s_c, s_x
        if (tid < 48) s_c[tid] = nxt;
        __syncthreads();
        const int64_t pn = p + gridDim.x;
        if (tid < 48 && pn < a.n) nxt = load_elem(a.ctrl, a.dtype, pn * 48 + tid);
        for (int e = tid; e < nu * 12; e += kTensorThreads) {
            const int row = e / 12, jk = e - row * 12;
            const float* bu = s_bu + row * 4;
            float x = bu[0] * s_c[jk];
            x = fmaf(bu[1], s_c[12 + jk], x);
            x = fmaf(bu[2], s_c[24 + jk], x);
            x = fmaf(bu[3], s_c[36 + jk], x);
            s_x[e] = x;
        }
        __syncthreads();
        float4* out = reinterpret_cast<float4*>(a.out + p * pts * 3);
        for (int q = tid; q < n_quads; q += kTensorThreads) {
            const int row = q / quads_per_row;
            const int b0 = (q - row * quads_per_row) * 4;
            const float* X = s_x + row * 12;
            float r[12];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const float4 bv = s_bv[b0 + m];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    float v = bv.x * X[k];
                    v = fmaf(bv.y, X[3 + k], v);
                    v = fmaf(bv.z, X[6 + k], v);
                    v = fmaf(bv.w, X[9 + k], v);
                    r[m * 3 + k] = v;
                }
            }
            float4* o = out + ((int64_t)row * nv + b0) * 3 / 4;
            o[0] = make_float4(r[0], r[1], r[2], r[3]);
            o[1] = make_float4(r[4], r[5], r[6], r[7]);
            o[2] = make_float4(r[8], r[9], r[10], r[11]);
        }
    }
}

// Fast path for small grids (nu <= 64, nv a multiple of 4): one warp per
// patch, no block barrier after the tables.  Lane l builds the isoline
// control points X[a] of rows a = l, l + 32 (12 floats each), then the warp
// sweeps the grid one row of up to 32 points at a time: lane l evaluates
// point (a, b0 + l) with Bv[b0 + l] held in registers, stages its 3 floats in
// a warp-private buffer and 24 lanes write the 384-byte row segment as float4.
__global__ void __launch_bounds__(kSurfWarps * 32, 5) k_surface_bicubic3_warp(const TensorArgs a)
{
    __shared__ float4 s_bv[kTensorMaxGrid];                   // Bv[b][0..3]
    __shared__ float4 s_bu[kSurfMaxRows];                     // Bu[a][0..3]
    __shared__ float4 s_x[kSurfWarps][kSurfMaxRows * 3];      // X[a][j][k], 12 floats per row
    __shared__ float4 s_st[kSurfWarps][2][24];                // 32 points x 3 floats, two buffers
    __shared__ float4 s_c4[kSurfWarps][12];                   // C[i][j][k]
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    bernstein_table(reinterpret_cast<float*>(s_bu), a.nu, 3, tid, kSurfWarps * 32);
    bernstein_table(reinterpret_cast<float*>(s_bv), a.nv, 3, tid, kSurfWarps * 32);
    __syncthreads();

    const int nu = a.nu, nv = a.nv;
    const int64_t pts = (int64_t)nu * nv;
    const int64_t stride = (int64_t)gridDim.x * kSurfWarps;
    int64_t p = (int64_t)blockIdx.x * kSurfWarps + w;
    float c0 = 0.f, c1 = 0.f;   // this lane's control-point elements, l and 32 + l
    if (p < a.n) {
        c0 = load_elem(a.ctrl, a.dtype, p * 48 + lane);
        if (lane < 16) c1 = load_elem(a.ctrl, a.dtype, p * 48 + 32 + lane);
    }
    float* cw = reinterpret_cast<float*>(s_c4[w]);
    int buf = 0;
    for (; p < a.n; p += stride) {
        __syncwarp();  // the previous patch is done with s_c and s_x
        cw[lane] = c0;
        if (lane < 16) cw[32 + lane] = c1;
        __syncwarp();
        const int64_t pn = p + stride;  // the next patch of this warp, loaded while this one runs
        if (pn < a.n) {
            c0 = load_elem(a.ctrl, a.dtype, pn * 48 + lane);
            if (lane < 16) c1 = load_elem(a.ctrl, a.dtype, pn * 48 + 32 + lane);
        }
        const float4* cw4 = reinterpret_cast<const float4*>(cw);   // C[i][4q..4q+3] = cw4[3 i + q]
#pragma unroll 1
        for (int q = 0; q < 3; ++q) {   // columns 4q..4q+3 of the 12 per row
            const float4 k0 = cw4[q], k1 = cw4[3 + q], k2 = cw4[6 + q], k3 = cw4[9 + q];
            for (int row = lane; row < nu; row += 32) {
                const float4 bu = s_bu[row];
                float4 x;
                x.x = fmaf(bu.w, k3.x, fmaf(bu.z, k2.x, fmaf(bu.y, k1.x, bu.x * k0.x)));
                x.y = fmaf(bu.w, k3.y, fmaf(bu.z, k2.y, fmaf(bu.y, k1.y, bu.x * k0.y)));
                x.z = fmaf(bu.w, k3.z, fmaf(bu.z, k2.z, fmaf(bu.y, k1.z, bu.x * k0.z)));
                x.w = fmaf(bu.w, k3.w, fmaf(bu.z, k2.w, fmaf(bu.y, k1.w, bu.x * k0.w)));
                s_x[w][row * 3 + q] = x;
            }
        }
        __syncwarp();
        float4* out = reinterpret_cast<float4*>(a.out + p * pts * 3);
        for (int b0 = 0; b0 < nv; b0 += 32) {
            const int b = b0 + lane;
            const float4 bv = b < nv ? s_bv[b] : make_float4(0.f, 0.f, 0.f, 0.f);
            const int nvec = min(32, nv - b0) * 3 / 4;   // float4 per row segment
#pragma unroll 2
            for (int row = 0; row < nu; ++row) {
                const float4 x0 = s_x[w][row * 3], x1 = s_x[w][row * 3 + 1], x2 = s_x[w][row * 3 + 2];
                // X[row][j][k] sits at float 3 j + k of the row
                float P0 = bv.x * x0.x, P1 = bv.x * x0.y, P2 = bv.x * x0.z;
                P0 = fmaf(bv.y, x0.w, P0);
                P1 = fmaf(bv.y, x1.x, P1);
                P2 = fmaf(bv.y, x1.y, P2);
                P0 = fmaf(bv.z, x1.z, P0);
                P1 = fmaf(bv.z, x1.w, P1);
                P2 = fmaf(bv.z, x2.x, P2);
                P0 = fmaf(bv.w, x2.y, P0);
                P1 = fmaf(bv.w, x2.z, P1);
                P2 = fmaf(bv.w, x2.w, P2);
                float* st = reinterpret_cast<float*>(s_st[w][buf]);
                st[lane * 3 + 0] = P0;
                st[lane * 3 + 1] = P1;
                st[lane * 3 + 2] = P2;
                __syncwarp();
                if (lane < nvec) out[((int64_t)row * nv + b0) * 3 / 4 + lane] = s_st[w][buf][lane];
                buf ^= 1;   // the next row stages in the other buffer, so no second barrier
            }
        }
    }
}

// General surfaces: any degrees <= 7, dim 1..4, grid <= 256 per axis.  One
// thread per output point (strided), outputs staged in shared memory and
// written as consecutive floats.
__global__ void __launch_bounds__(kTensorThreads) k_surface_generic(const TensorArgs a)
{
    extern __shared__ float sm[];
    const int du = a.du, dv = a.dv, dim = a.dim, nu = a.nu, nv = a.nv;
    float* s_bu = sm;                                   // nu * (du+1)
    float* s_bv = s_bu + nu * (du + 1);                 // nv * (dv+1)
    float* s_c = s_bv + nv * (dv + 1);                  // (du+1)(dv+1)dim
    float* s_x = s_c + (du + 1) * (dv + 1) * dim;       // nu * (dv+1) * dim
    float* s_o = s_x + nu * (dv + 1) * dim;             // kTensorThreads * dim
    const int tid = threadIdx.x;
    bernstein_table(s_bu, nu, du, tid, kTensorThreads);
    bernstein_table(s_bv, nv, dv, tid, kTensorThreads);
    const int per = (du + 1) * (dv + 1) * dim;
    const int64_t pts = (int64_t)nu * nv;
    for (int64_t p = blockIdx.x; p < a.n; p += gridDim.x) {
        __syncthreads();
        for (int e = tid; e < per; e += kTensorThreads) s_c[e] = load_elem(a.ctrl, a.dtype, p * per + e);
        __syncthreads();
        const int xr = (dv + 1) * dim;
        for (int e = tid; e < nu * xr; e += kTensorThreads) {
            const int row = e / xr, jk = e - row * xr;
            float x = 0.f;
            for (int i = 0; i <= du; ++i) x = fmaf(s_bu[row * (du + 1) + i], s_c[i * xr + jk], x);
            s_x[e] = x;
        }
        __syncthreads();
        float* out = a.out + p * pts * dim;
        for (int64_t q0 = 0; q0 < pts; q0 += kTensorThreads) {
            const int64_t q = q0 + tid;
            if (q < pts) {
                const int row = (int)(q / nv), b = (int)(q - (int64_t)row * nv);
                for (int k = 0; k < dim; ++k) {
                    float v = 0.f;
                    for (int j = 0; j <= dv; ++j) v = fmaf(s_bv[b * (dv + 1) + j], s_x[row * xr + j * dim + k], v);
                    s_o[tid * dim + k] = v;
                }
            }
            __syncthreads();
            const int64_t valid = min((int64_t)kTensorThreads, pts - q0) * dim;
            for (int f = tid; f < valid; f += kTensorThreads) out[q0 * dim + f] = s_o[f];
            __syncthreads();
        }
    }
}

// Volumes (any degrees <= 7, dim 1..4): Y and Z stages in shared memory, one
// thread per (a, b) line writing its nw * dim consecutive values.
__global__ void __launch_bounds__(kTensorThreads) k_volume(const TensorArgs a)
{
    extern __shared__ float sm[];
    const int du = a.du, dv = a.dv, dw = a.dw, dim = a.dim, nu = a.nu, nv = a.nv, nw = a.nw;
    float* s_bu = sm;
    float* s_bv = s_bu + nu * (du + 1);
    float* s_bw = s_bv + nv * (dv + 1);
    float* s_c = s_bw + nw * (dw + 1);
    const int per = (du + 1) * (dv + 1) * (dw + 1) * dim;
    float* s_y = s_c + per;                                 // nu (dv+1) (dw+1) dim
    float* s_z = s_y + nu * (dv + 1) * (dw + 1) * dim;      // nu nv (dw+1) dim
    const int tid = threadIdx.x;
    bernstein_table(s_bu, nu, du, tid, kTensorThreads);
    bernstein_table(s_bv, nv, dv, tid, kTensorThreads);
    bernstein_table(s_bw, nw, dw, tid, kTensorThreads);
    const int lk = (dw + 1) * dim;                          // (l, k) entries of one (i, j)
    const int64_t pts = (int64_t)nu * nv * nw;
    for (int64_t p = blockIdx.x; p < a.n; p += gridDim.x) {
        __syncthreads();
        for (int e = tid; e < per; e += kTensorThreads) s_c[e] = load_elem(a.ctrl, a.dtype, p * per + e);
        __syncthreads();
        const int ny = nu * (dv + 1) * lk;
        for (int e = tid; e < ny; e += kTensorThreads) {
            const int row = e / ((dv + 1) * lk), jlk = e - row * ((dv + 1) * lk);
            float y = 0.f;
            for (int i = 0; i <= du; ++i) y = fmaf(s_bu[row * (du + 1) + i], s_c[i * (dv + 1) * lk + jlk], y);
            s_y[e] = y;
        }
        __syncthreads();
        const int nz = nu * nv * lk;
        for (int e = tid; e < nz; e += kTensorThreads) {
            const int ab = e / lk, l_k = e - ab * lk;
            const int ai = ab / nv, b = ab - ai * nv;
            float z = 0.f;
            for (int j = 0; j <= dv; ++j)
                z = fmaf(s_bv[b * (dv + 1) + j], s_y[(ai * (dv + 1) + j) * lk + l_k], z);
            s_z[e] = z;
        }
        __syncthreads();
        float* out = a.out + p * pts * dim;
        const int line = nw * dim;
        if (line % 4 == 0 && (((uintptr_t)out) & 15) == 0) {
            // one thread per (a, b) line: its nw * dim values as float4 stores
            for (int ab = tid; ab < nu * nv; ab += kTensorThreads) {
                float4* o = reinterpret_cast<float4*>(out + (int64_t)ab * line);
                const float* z = s_z + ab * lk;
                for (int f4 = 0; f4 < line / 4; ++f4) {
                    float r[4];
                    for (int m = 0; m < 4; ++m) {
                        const int ck = f4 * 4 + m, c = ck / dim, k = ck - c * dim;
                        float v = 0.f;
                        for (int l = 0; l <= dw; ++l) v = fmaf(s_bw[c * (dw + 1) + l], z[l * dim + k], v);
                        r[m] = v;
                    }
                    o[f4] = make_float4(r[0], r[1], r[2], r[3]);
                }
            }
        } else {
            for (int e = tid; e < nu * nv * line; e += kTensorThreads) {
                // consecutive threads write consecutive floats of the volume
                const int ab = e / line, ck = e - ab * line;
                const int c = ck / dim, k = ck - c * dim;
                float v = 0.f;
                for (int l = 0; l <= dw; ++l) v = fmaf(s_bw[c * (dw + 1) + l], s_z[ab * lk + l * dim + k], v);
                out[e] = v;
            }
        }
    }
}

size_t tensor_smem_bytes(const TensorArgs& a)
{
    if (a.dw < 0) {
        return sizeof(float) * ((size_t)a.nu * (a.du + 1) + (size_t)a.nv * (a.dv + 1) +
                                (size_t)(a.du + 1) * (a.dv + 1) * a.dim + (size_t)a.nu * (a.dv + 1) * a.dim +
                                (size_t)kTensorThreads * a.dim);
    }
    const size_t lk = (size_t)(a.dw + 1) * a.dim;
    return sizeof(float) * ((size_t)a.nu * (a.du + 1) + (size_t)a.nv * (a.dv + 1) + (size_t)a.nw * (a.dw + 1) +
                            (size_t)(a.du + 1) * (a.dv + 1) * lk + (size_t)a.nu * (a.dv + 1) * lk +
                            (size_t)a.nu * a.nv * lk);
}

static TensorArgs to_args(const TensorLaunch& t)
{
    TensorArgs a;
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
    a.vparts = 1;
    return a;
}

size_t tensor_product_smem(const TensorLaunch& t) { return tensor_smem_bytes(to_args(t)); }

LaunchResult launch_tensor_product(const TensorLaunch& t, cudaStream_t s, const LaunchHooks& h)
{
    TensorArgs a = to_args(t);
    const void* kern;
    size_t smem = 0;
    int threads = kTensorThreads;
    int64_t work = a.n;
    const bool bicubic3 = a.dw < 0 && a.du == 3 && a.dv == 3 && a.dim == 3 && a.nv % 4 == 0 &&
                          ((uintptr_t)a.out & 15) == 0;
    const bool tricubic1 = a.dw == 3 && a.du == 3 && a.dv == 3 && a.dim == 1 && a.nu <= kVolMaxRows &&
                           a.nw % 4 == 0 && ((uintptr_t)a.out & 15) == 0;
    if (bicubic3 && a.nu <= kSurfMaxRows) {
        kern = (const void*)k_surface_bicubic3_warp;
        threads = kSurfWarps * 32;
        work = (a.n + kSurfWarps - 1) / kSurfWarps;
    } else if (tricubic1) {
        kern = (const void*)k_volume_tricubic1_warp<VOL_U_CORES>;
        threads = kSurfWarps * 32;
        a.vparts = volume_parts(a.n, a.nu, h.sm_count);
        work = (a.n * a.vparts + kSurfWarps - 1) / kSurfWarps;
    } else if (bicubic3) {
        kern = (const void*)k_surface_bicubic3;
    } else {
        kern = a.dw < 0 ? (const void*)k_surface_generic : (const void*)k_volume;
        smem = tensor_smem_bytes(a);
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return {0, e};
        }
    }
    const int grid = persistent_grid(kern, threads, smem, h.sm_count, work);
    const SurfTexArgs no_tex{};  // the CUDA-core volume kernel reads no texture
    void* args[] = {(void*)&a, (void*)&no_tex};
    h.count(h.self);
    h.begin(h.self, s);
    cudaError_t e = cudaLaunchKernel(kern, dim3(grid), dim3(threads), args, smem, s);
    h.end(h.self, s);
    return {1, e};
}

}  // namespace bez
