// grad.cu -- adjoint of (rational) Bezier curve evaluation.
//
// For curves C(t) = A(t) / W(t), A = sum_i B_i(t) w_i P_i, W = sum_i B_i(t) w_i
// (w = 1 for integral curves) and an upstream gradient g_j = dL/dC(t_j):
//   dL/dP_i = sum_j (w_i B_i(t_j) / W_j) g_j
//   dL/dw_i = sum_j B_i(t_j) (P_i - C_j) . g_j / W_j
//   dL/dt_j = g_j . (A'(t_j) - C_j W'(t_j)) / W_j      (0 where t was clamped)
// with A' = d sum_i B_i^(d-1) (w_(i+1) P_(i+1) - w_i P_i) and W' likewise.
// The Bernstein values come from the basis triangle B^(r)_i = (1-t) B^(r-1)_i
// + t B^(r-1)_(i-1), whose level d-1 gives the derivative basis.
//
// Fused squared error (target given): g_j = 2 s (C(t_j) - target_j) is formed
// in the kernel from the curve value it computes anyway, and the per-curve
// loss s sum_j ||C(t_j) - target_j||^2 is summed alongside, so a fitting step
// reads t and the targets once and writes dt (no point or gradient arrays).
//
// One warp per curve; lanes take samples j = lane + 32 m (coalesced reads of
// t and g), two at a time (j and j + 32: independent arithmetic to
// interleave), keep per-lane partial sums of the per-curve gradients in
// registers, and combine them at the end of the curve (one 16-value
// reduce-scatter for fixed degrees, butterflies otherwise).  Per-sample dt is
// written directly (per-curve t) or summed over curves (shared t) in shared
// memory and then with one global atomic per block and parameter.  The next
// pair's loads are issued before the current pair's arithmetic, and the
// output mode is decided once per launch, outside the sample loop.
//
// Per curve the homogeneous points q_i = w_i P_i and the scaled differences
// d (q_(i+1) - q_i), d (w_(i+1) - w_i) are formed once, so a sample costs the
// basis triangle plus one FMA per (point, coordinate) for each of A, A' and
// dL/dP.  Integral curves (RAT false) drop W, W', the division and the weight
// sums: C = A exactly as the Bernstein sum.
#include "curve_eval.cuh"

namespace bez {

constexpr int kGradMaxDim = 4;

// samples per loop iteration: two independent samples to interleave while
// the pair's registers fit, one for high degrees
__host__ __device__ constexpr int grad_pair(int D, bool RAT) { return (D >= 1 && D <= (RAT ? 3 : 4)) ? 2 : 1; }

// resident blocks per SM the register budget is sized for (64, 80 or 128
// registers a thread at 256 threads a block)
__host__ __device__ constexpr int grad_min_blocks(int D, bool RAT)
{
    return D == 0 ? 2 : grad_pair(D, RAT) == 1 ? (!RAT && D <= 5 ? 3 : 2) : (!RAT && D <= 3) ? 4 : 2;
}

// dL/dt output: none, per-curve array, or shared t summed over curves with
// atomics into gt_sum (this block's shared-memory partial sums, or the global
// array when n_t is too large for shared memory)
enum { GT_NONE = 0, GT_PER_CURVE = 1, GT_SHARED = 2 };

// One curve's state in a lane: control data and the lane's partial sums.
template <int D, int DIM, bool RAT>
struct GradCurve {
    static constexpr int N = Deg<D>::N;
    static constexpr int M = DIM ? DIM : kGradMaxDim;
    int d, dim;
    float P[N][M], w[N], dq[N][M], dw[N];
    float acc_c[N][M], acc_w[N], loss;

    __device__ __forceinline__ void setup(const GradArgs& a, int64_t c)
    {
        d = Deg<D>::get(a.degree);
        dim = DIM ? DIM : a.dim;
        const int dd = D ? D : d;  // a constant bound unrolls; the runtime degree loops
        float q[N][M];
#pragma unroll
        for (int i = 0; i <= dd; ++i) {
            w[i] = RAT ? __ldg(a.weights + c * (d + 1) + i) : 1.f;
#pragma unroll
            for (int k = 0; k < M; ++k) {
                if (k >= dim) break;
                P[i][k] = __ldg(a.ctrl + (c * (d + 1) + i) * dim + k);
                q[i][k] = RAT ? w[i] * P[i][k] : P[i][k];
            }
        }
        const float fd = (float)d;
#pragma unroll
        for (int i = 0; i < dd; ++i) {
            if (RAT) dw[i] = fd * (w[i + 1] - w[i]);
#pragma unroll
            for (int k = 0; k < M; ++k) {
                if (k >= dim) break;
                dq[i][k] = fd * (q[i + 1][k] - q[i][k]);
            }
        }
#pragma unroll
        for (int i = 0; i <= dd; ++i) {
            acc_w[i] = 0.f;
#pragma unroll
            for (int k = 0; k < M; ++k) acc_c[i][k] = 0.f;
        }
        loss = 0.f;
    }

    // One sample: accumulate its dL/dP, dL/dw (and loss) terms; return dL/dt.
    // FUSED: v is the target and g = g2 (C - v) mask; else v is g.  A sample
    // past the end arrives with mask 0 (fused) or v = 0, and adds nothing.
    template <bool FUSED>
    __device__ __forceinline__ float sample(float traw, const float (&v)[M], float mask, float g2)
    {
        const int dd = D ? D : d;
        const float t = clamp01(traw);
        const float s = 1.0f - t;
        // basis triangle; keep level d-1 for the derivative
        float B[N], Bd[N];
        B[0] = 1.f;
#pragma unroll
        for (int r = 1; r <= dd; ++r) {
            if (r == dd) {
#pragma unroll
                for (int i = 0; i < dd; ++i) Bd[i] = B[i];
            }
            B[r] = t * B[r - 1];
#pragma unroll
            for (int i = r - 1; i >= 1; --i) B[i] = fmaf(t, B[i - 1], s * B[i]);
            B[0] = s * B[0];
        }
        float A[M], dA[M];
        float W = RAT ? 0.f : 1.f, dW = 0.f;
#pragma unroll
        for (int k = 0; k < M; ++k) A[k] = dA[k] = 0.f;
#pragma unroll
        for (int i = 0; i <= dd; ++i) {
            const float bw = RAT ? B[i] * w[i] : B[i];
            if (RAT) W += bw;
#pragma unroll
            for (int k = 0; k < M; ++k)
                if (k < dim) A[k] = fmaf(bw, P[i][k], A[k]);
        }
#pragma unroll
        for (int i = 0; i < dd; ++i) {
            if (RAT) dW = fmaf(Bd[i], dw[i], dW);
#pragma unroll
            for (int k = 0; k < M; ++k)
                if (k < dim) dA[k] = fmaf(Bd[i], dq[i][k], dA[k]);
        }
        const float invW = RAT ? __frcp_rn(W) : 1.f;
        float C[M], gj[M];
#pragma unroll
        for (int k = 0; k < M; ++k) {
            C[k] = RAT ? A[k] * invW : A[k];
            if (FUSED) {
                // fused squared error: g = 2 s (C - target), loss += ||C - target||^2
                const float r = (C[k] - v[k]) * mask;
                gj[k] = g2 * r;
                if (k < dim) loss = fmaf(r, r, loss);
            } else {
                gj[k] = v[k];
            }
        }
#pragma unroll
        for (int i = 0; i <= dd; ++i) {
            const float f = RAT ? B[i] * w[i] * invW : B[i];
#pragma unroll
            for (int k = 0; k < M; ++k)
                if (k < dim) acc_c[i][k] = fmaf(f, gj[k], acc_c[i][k]);
            if (RAT) {
                float dot = 0.f;
#pragma unroll
                for (int k = 0; k < M; ++k)
                    if (k < dim) dot = fmaf(P[i][k] - C[k], gj[k], dot);
                acc_w[i] = fmaf(B[i] * invW, dot, acc_w[i]);
            }
        }
        float gt = 0.f;
#pragma unroll
        for (int k = 0; k < M; ++k)
            if (k < dim) gt = fmaf(gj[k], RAT ? fmaf(-C[k], dW, dA[k]) : dA[k], gt);
        return (traw >= 0.f && traw <= 1.f) ? (RAT ? gt * invW : gt) : 0.f;  // clamped t: no dL/dt
    }

    // Per-curve sums over the warp.  Fixed degree and dim: the values
    // (dL/dP, dL/dw, loss) go through one 16-value reduce-scatter, lane 2e
    // writing value e, and any beyond 16 through butterflies; otherwise one
    // butterfly per value, lane e writing element e.
    __device__ __forceinline__ void finish(const GradArgs& a, int64_t c, int lane)
    {
        if constexpr (D > 0 && DIM > 0) {
            constexpr int NC = N * M;                      // dL/dP values
            constexpr int NV = NC + (RAT ? N : 0) + 1;     // + dL/dw + loss
            float v[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                float x = 0.f;
                if (e < NC) x = acc_c[e / M][e % M];
                else if (RAT && e < NC + N) x = acc_w[e - NC];
                else if (e == NV - 1) x = loss;
                v[e] = x;
            }
            const float tot = warp_sum16_scatter(v, lane);
            const int e = (lane >> 1) & 15;
            if ((lane & 1) == 0) {
                if (e < NC) {
                    if (a.grad_ctrl) a.grad_ctrl[c * NC + e] = tot;
                } else if (RAT && e < NC + N) {
                    if (a.grad_w) a.grad_w[c * N + (e - NC)] = tot;
                } else if (e == NV - 1 && a.loss) {
                    a.loss[c] = a.loss_scale * tot;
                }
            }
            if constexpr (NV > 16) {
                // values 16.. (at most 16 more here): one butterfly each
#pragma unroll
                for (int e2 = 16; e2 < NV; ++e2) {
                    float x = e2 < NC ? acc_c[e2 / M][e2 % M] : (RAT && e2 < NC + N) ? acc_w[e2 - NC] : loss;
                    x = warp_sum(x);
                    if (lane == 0) {
                        if (e2 < NC) {
                            if (a.grad_ctrl) a.grad_ctrl[c * NC + e2] = x;
                        } else if (RAT && e2 < NC + N) {
                            if (a.grad_w) a.grad_w[c * N + (e2 - NC)] = x;
                        } else if (a.loss) {
                            a.loss[c] = a.loss_scale * x;
                        }
                    }
                }
            }
            return;
        }
        const int nc = (d + 1) * dim;
        const int dd = D ? D : d;
#pragma unroll
        for (int i = 0; i <= dd; ++i) {
#pragma unroll
            for (int k = 0; k < M; ++k) {
                if (k >= dim) break;
                const float v = warp_sum(acc_c[i][k]);
                if (a.grad_ctrl && lane == (i * dim + k) % 32) a.grad_ctrl[c * nc + i * dim + k] = v;
            }
            if (RAT) {
                const float vw = warp_sum(acc_w[i]);
                if (a.grad_w && lane == i % 32) a.grad_w[c * (d + 1) + i] = vw;
            }
        }
        if (a.loss) {
            const float l = warp_sum(loss);
            if (lane == 0) a.loss[c] = a.loss_scale * l;
        }
    }
};

// read-only load asking L2 to fetch the whole 256-byte block around the
// address, so that a warp's streaming reads of t and the targets bring the
// next rows into L2 with the current ones
__device__ __forceinline__ float ld_stream(const float* p)
{
    float v;
    asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

template <int M>
__device__ __forceinline__ void load_sample(const float* tc, const float* vc, int dim, int n_t, int j, float& t,
                                            float (&v)[M])
{
    t = 0.f;
#pragma unroll
    for (int k = 0; k < M; ++k) v[k] = 0.f;
    if (j < n_t) {
        t = ld_stream(tc + j);
#pragma unroll
        for (int k = 0; k < M; ++k)
            if (k < dim) v[k] = ld_stream(vc + j * dim + k);
    }
}

template <int GTM>
__device__ __forceinline__ void put_gt(float* gtc, float* gt_sum, int j, float gt)
{
    if (GTM == GT_PER_CURVE) gtc[j] = gt;
    else if (GTM == GT_SHARED) atomicAdd(gt_sum + j, gt);
}

template <int D, int DIM, bool RAT, bool FUSED, int GTM>
__device__ __forceinline__ void grad_curves(const GradArgs& a, float* gt_sum)
{
    using G = GradCurve<D, DIM, RAT>;
    constexpr int M = G::M;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int n_t = a.n_t;
    const int dim = DIM ? DIM : a.dim;
    const float* vsrc = FUSED ? a.target : a.g;
    const float g2 = 2.0f * a.loss_scale;
    const int64_t n_warps = (int64_t)gridDim.x * kWarps;
    for (int64_t c = (int64_t)blockIdx.x * kWarps + wib; c < a.n_curves; c += n_warps) {
        G e;
        e.setup(a, c);
        const float* tc = a.t + c * a.t_stride;
        const float* vc = vsrc + c * (int64_t)n_t * dim;
        float* gtc = GTM == GT_PER_CURVE ? a.grad_t + c * (int64_t)n_t : nullptr;
        if constexpr (grad_pair(D, RAT) == 2) {
            float tA, tB, vA[M], vB[M];
            load_sample<M>(tc, vc, dim, n_t, lane, tA, vA);
            load_sample<M>(tc, vc, dim, n_t, lane + 32, tB, vB);
            for (int j = lane; j < n_t; j += 64) {
                const float t0 = tA, t1 = tB;
                float v0[M], v1[M];
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    v0[k] = vA[k];
                    v1[k] = vB[k];
                }
                load_sample<M>(tc, vc, dim, n_t, j + 64, tA, vA);
                load_sample<M>(tc, vc, dim, n_t, j + 96, tB, vB);
                const bool has1 = j + 32 < n_t;
                const float gt0 = e.template sample<FUSED>(t0, v0, 1.f, g2);
                const float gt1 = e.template sample<FUSED>(t1, v1, has1 ? 1.f : 0.f, g2);
                put_gt<GTM>(gtc, gt_sum, j, gt0);
                if (has1) put_gt<GTM>(gtc, gt_sum, j + 32, gt1);
            }
        } else {
            float tA, vA[M];
            load_sample<M>(tc, vc, dim, n_t, lane, tA, vA);
            for (int j = lane; j < n_t; j += 32) {
                const float t0 = tA;
                float v0[M];
#pragma unroll
                for (int k = 0; k < M; ++k) v0[k] = vA[k];
                load_sample<M>(tc, vc, dim, n_t, j + 32, tA, vA);
                put_gt<GTM>(gtc, gt_sum, j, e.template sample<FUSED>(t0, v0, 1.f, g2));
            }
        }
        e.finish(a, c, lane);
    }
}

template <int D, int DIM, bool RAT>
__global__ void __launch_bounds__(kWarps * 32, grad_min_blocks(D, RAT)) k_grad(const GradArgs a)
{
    extern __shared__ float s_gt[];  // shared-t dL/dt partial sums of this block
    const int gtm = !a.grad_t ? GT_NONE : a.t_stride ? GT_PER_CURVE : GT_SHARED;
    const bool smem_sum = gtm == GT_SHARED && a.shared_gt;
    float* gt_sum = smem_sum ? s_gt : a.grad_t;
    if (smem_sum) {
        for (int j = threadIdx.x; j < a.n_t; j += blockDim.x) s_gt[j] = 0.f;
        __syncthreads();
    }
    if (a.target) {
        if (gtm == GT_NONE) grad_curves<D, DIM, RAT, true, GT_NONE>(a, gt_sum);
        else if (gtm == GT_PER_CURVE) grad_curves<D, DIM, RAT, true, GT_PER_CURVE>(a, gt_sum);
        else grad_curves<D, DIM, RAT, true, GT_SHARED>(a, gt_sum);
    } else {
        if (gtm == GT_NONE) grad_curves<D, DIM, RAT, false, GT_NONE>(a, gt_sum);
        else if (gtm == GT_PER_CURVE) grad_curves<D, DIM, RAT, false, GT_PER_CURVE>(a, gt_sum);
        else grad_curves<D, DIM, RAT, false, GT_SHARED>(a, gt_sum);
    }
    if (smem_sum) {
        __syncthreads();
        for (int j = threadIdx.x; j < a.n_t; j += blockDim.x) atomicAdd(a.grad_t + j, s_gt[j]);
    }
}

template <bool RAT>
static const void* grad_kernel(int degree, int dim)
{
    if (dim == 3) {
        switch (degree) {
        case 1: return (const void*)k_grad<1, 3, RAT>;
        case 2: return (const void*)k_grad<2, 3, RAT>;
        case 3: return (const void*)k_grad<3, 3, RAT>;
        case 4: return (const void*)k_grad<4, 3, RAT>;
        case 5: return (const void*)k_grad<5, 3, RAT>;
        case 6: return (const void*)k_grad<6, 3, RAT>;
        case 7: return (const void*)k_grad<7, 3, RAT>;
        default: break;
        }
    }
    return (const void*)k_grad<0, 0, RAT>;
}

LaunchResult launch_grad(const GradArgs& a, cudaStream_t s, const LaunchHooks& h)
{
    const void* kern = a.weights ? grad_kernel<true>(a.degree, a.dim) : grad_kernel<false>(a.degree, a.dim);
    const size_t smem = (a.t_stride == 0 && a.grad_t && a.shared_gt) ? (size_t)a.n_t * sizeof(float) : 0;
    const int grid = persistent_grid(kern, kWarps * 32, smem, h.sm_count, (a.n_curves + kWarps - 1) / kWarps);
    void* args[] = {(void*)&a};
    h.count(h.self);
    h.begin(h.self, s);
    cudaError_t e = cudaLaunchKernel(kern, dim3(grid), dim3(kWarps * 32), args, smem, s);
    h.end(h.self, s);
    return {1, e};
}

}  // namespace bez
