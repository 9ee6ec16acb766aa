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
// t and g), keep per-lane partial sums of the per-curve gradients in
// registers, and combine them with a butterfly of shuffles.  Per-sample dt is
// written directly (per-curve t) or summed over curves (shared t) in shared
// memory and then with one global atomic per block and parameter.
//
// Per curve the homogeneous points q_i = w_i P_i and the scaled differences
// d (q_(i+1) - q_i), d (w_(i+1) - w_i) are formed once, so a sample costs the
// basis triangle plus one FMA per (point, coordinate) for each of A, A' and
// dL/dP.  Integral curves (RAT false) drop W, W', the division and the weight
// sums: C = A exactly as the Bernstein sum.  The next sample's loads are
// issued before the current sample's arithmetic.
#include "curve_eval.cuh"

namespace bez {

constexpr int kGradMaxDim = 4;

// resident blocks per SM the register budget is sized for (64, 80 or 128
// registers a thread at 256 threads a block)
__host__ __device__ constexpr int grad_min_blocks(int D, bool RAT)
{
    return D == 0 ? 2 : (!RAT && D <= 4) ? 4 : (D <= 3 || (!RAT && D <= 5)) ? 3 : 2;
}

template <int D, int DIM, bool RAT>
__global__ void __launch_bounds__(kWarps * 32, grad_min_blocks(D, RAT)) k_grad(const GradArgs a)
{
    constexpr int N = Deg<D>::N;
    constexpr int M = DIM ? DIM : kGradMaxDim;
    constexpr int kUnrollN = D ? N : 1;  // runtime degree: loops, arrays in local memory
    extern __shared__ float s_gt[];  // shared-t dL/dt partial sums of this block
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int d = Deg<D>::get(a.degree);
    const int dim = DIM ? DIM : a.dim;
    const bool shared_t = a.t_stride == 0;
    const bool fused = a.target != nullptr;
    const float* gsrc = fused ? a.target : a.g;  // per-sample vector input
    const float g2 = 2.0f * a.loss_scale;
    const int n_t = a.n_t;
    if (shared_t && a.grad_t && a.shared_gt) {
        for (int j = threadIdx.x; j < n_t; j += blockDim.x) s_gt[j] = 0.f;
        __syncthreads();
    }
    const int64_t n_warps = (int64_t)gridDim.x * kWarps;
    for (int64_t c = (int64_t)blockIdx.x * kWarps + wib; c < a.n_curves; c += n_warps) {
        // q_i = w_i P_i; dq_i = d (q_(i+1) - q_i); dw_i = d (w_(i+1) - w_i)
        float P[N][M], q[N][M], w[N], dq[N][M], dw[N];
#pragma unroll kUnrollN
        for (int i = 0; i < N; ++i) {
            if (i > d) break;
            w[i] = RAT ? __ldg(a.weights + c * (d + 1) + i) : 1.f;
#pragma unroll
            for (int k = 0; k < M; ++k) {
                if (k >= dim) break;
                P[i][k] = __ldg(a.ctrl + (c * (d + 1) + i) * dim + k);
                q[i][k] = RAT ? w[i] * P[i][k] : P[i][k];
            }
        }
        const float fd = (float)d;
#pragma unroll kUnrollN
        for (int i = 0; i < N - 1; ++i) {
            if (i >= d) break;
            if (RAT) dw[i] = fd * (w[i + 1] - w[i]);
#pragma unroll
            for (int k = 0; k < M; ++k) {
                if (k >= dim) break;
                dq[i][k] = fd * (q[i + 1][k] - q[i][k]);
            }
        }
        float acc_c[N][M], acc_w[N];
        float loss_acc = 0.f;
#pragma unroll kUnrollN
        for (int i = 0; i < N; ++i) {
            acc_w[i] = 0.f;
#pragma unroll
            for (int k = 0; k < M; ++k) acc_c[i][k] = 0.f;
        }
        const float* tc = a.t + c * a.t_stride;
        const float* gc = gsrc + c * (int64_t)n_t * dim;
        // prefetched inputs of sample j
        float t_next = 0.f, v_next[M];
#pragma unroll
        for (int k = 0; k < M; ++k) v_next[k] = 0.f;
        if (lane < n_t) {
            t_next = __ldg(tc + lane);
#pragma unroll
            for (int k = 0; k < M; ++k)
                if (k < dim) v_next[k] = __ldg(gc + (int64_t)lane * dim + k);
        }
        for (int j = lane; j < n_t; j += 32) {
            const float traw = t_next;
            float v[M];
#pragma unroll
            for (int k = 0; k < M; ++k) v[k] = v_next[k];
            if (j + 32 < n_t) {
                t_next = __ldg(tc + j + 32);
#pragma unroll
                for (int k = 0; k < M; ++k)
                    if (k < dim) v_next[k] = __ldg(gc + (int64_t)(j + 32) * dim + k);
            }
            const float t = clamp01(traw);
            const float s = 1.0f - t;
            // basis triangle; keep level d-1 for the derivative
            float B[N], Bd[N];
            B[0] = 1.f;
#pragma unroll kUnrollN
            for (int r = 1; r < N; ++r) {
                if (r > d) break;
                if (r == d) {
#pragma unroll kUnrollN
                    for (int i = 0; i < N - 1; ++i)
                        if (i < d) Bd[i] = B[i];
                }
                B[r] = t * B[r - 1];
#pragma unroll
                for (int i = r - 1; i >= 1; --i) B[i] = fmaf(t, B[i - 1], s * B[i]);
                B[0] = s * B[0];
            }
            float A[M], dA[M];
            float W = 1.f, dW = 0.f;
#pragma unroll
            for (int k = 0; k < M; ++k) A[k] = dA[k] = 0.f;
            if (RAT) W = 0.f;
#pragma unroll kUnrollN
            for (int i = 0; i < N; ++i) {
                if (i > d) break;
                const float bw = RAT ? B[i] * w[i] : B[i];
                if (RAT) W += bw;
#pragma unroll
                for (int k = 0; k < M; ++k)
                    if (k < dim) A[k] = fmaf(bw, P[i][k], A[k]);
            }
#pragma unroll kUnrollN
            for (int i = 0; i < N - 1; ++i) {
                if (i >= d) break;
                if (RAT) dW = fmaf(Bd[i], dw[i], dW);
#pragma unroll
                for (int k = 0; k < M; ++k)
                    if (k < dim) dA[k] = fmaf(Bd[i], dq[i][k], dA[k]);
            }
            const float invW = RAT ? __frcp_rn(W) : 1.f;
            float C[M];
#pragma unroll
            for (int k = 0; k < M; ++k) C[k] = RAT ? A[k] * invW : A[k];
            float gj[M];
            if (fused) {
                // fused squared error: g = 2 s (C - target), loss += ||C - target||^2
#pragma unroll
                for (int k = 0; k < M; ++k) {
                    if (k >= dim) break;
                    const float r = C[k] - v[k];
                    gj[k] = g2 * r;
                    loss_acc = fmaf(r, r, loss_acc);
                }
            } else {
#pragma unroll
                for (int k = 0; k < M; ++k) gj[k] = v[k];
            }
#pragma unroll kUnrollN
            for (int i = 0; i < N; ++i) {
                if (i > d) break;
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
            if (a.grad_t) {
                float gt = 0.f;
#pragma unroll
                for (int k = 0; k < M; ++k)
                    if (k < dim) gt = fmaf(gj[k], RAT ? fmaf(-C[k], dW, dA[k]) : dA[k], gt);
                gt = (traw >= 0.f && traw <= 1.f) ? (RAT ? gt * invW : gt) : 0.f;
                if (!shared_t) a.grad_t[c * n_t + j] = gt;
                else if (a.shared_gt) atomicAdd(s_gt + j, gt);
                else atomicAdd(a.grad_t + j, gt);
            }
        }
        // butterfly: every lane ends with the curve's sums; lane e writes element e
        const int nc = (d + 1) * dim;
#pragma unroll kUnrollN
        for (int i = 0; i < N; ++i) {
            if (i > d) break;
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
            const float l = warp_sum(loss_acc);
            if (lane == 0) a.loss[c] = a.loss_scale * l;
        }
    }
    if (shared_t && a.grad_t && a.shared_gt) {
        __syncthreads();
        for (int j = threadIdx.x; j < n_t; j += blockDim.x) atomicAdd(a.grad_t + j, s_gt[j]);
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
