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
// One warp per curve; lanes take samples j = lane + 32 m (coalesced reads of
// t and g), keep per-lane partial sums of the per-curve gradients in
// registers, and combine them with a butterfly of shuffles.  Per-sample dt is
// written directly (per-curve t) or summed over curves (shared t) in shared
// memory and then with one global atomic per block and parameter.
#include "curve_eval.cuh"

namespace bez {

constexpr int kGradMaxDim = 4;

template <int D, int DIM>
__global__ void __launch_bounds__(kWarps * 32) k_grad(const GradArgs a)
{
    constexpr int N = Deg<D>::N;
    extern __shared__ float s_gt[];  // shared-t dL/dt partial sums of this block
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int d = Deg<D>::get(a.degree);
    const int dim = DIM ? DIM : a.dim;
    const bool rat = a.weights != nullptr;
    const bool shared_t = a.t_stride == 0;
    if (shared_t && a.grad_t && a.shared_gt) {
        for (int j = threadIdx.x; j < a.n_t; j += blockDim.x) s_gt[j] = 0.f;
        __syncthreads();
    }
    const int64_t n_warps = (int64_t)gridDim.x * kWarps;
    for (int64_t c = (int64_t)blockIdx.x * kWarps + wib; c < a.n_curves; c += n_warps) {
        // homogeneous control points q_i = (w_i P_i, w_i)
        float P[N][kGradMaxDim], w[N];
        for (int i = 0; i <= d; ++i) {
            w[i] = rat ? __ldg(a.weights + c * (d + 1) + i) : 1.f;
            for (int k = 0; k < dim; ++k) P[i][k] = __ldg(a.ctrl + (c * (d + 1) + i) * dim + k);
        }
        float acc_c[N][kGradMaxDim], acc_w[N];
        for (int i = 0; i <= d; ++i) {
            acc_w[i] = 0.f;
            for (int k = 0; k < dim; ++k) acc_c[i][k] = 0.f;
        }
        for (int j = lane; j < a.n_t; j += 32) {
            const float traw = __ldg(a.t + c * a.t_stride + j);
            const float t = clamp01(traw);
            const float s = 1.0f - t;
            // basis triangle; keep level d-1 for the derivative
            float B[N], Bd[N];
            B[0] = 1.f;
            for (int r = 1; r <= d; ++r) {
                if (r == d)
                    for (int i = 0; i < d; ++i) Bd[i] = B[i];
                B[r] = t * B[r - 1];
                for (int i = r - 1; i >= 1; --i) B[i] = fmaf(t, B[i - 1], s * B[i]);
                B[0] = s * B[0];
            }
            float gj[kGradMaxDim];
            for (int k = 0; k < dim; ++k) gj[k] = __ldg(a.g + (c * a.n_t + j) * dim + k);
            float A[kGradMaxDim], dA[kGradMaxDim];
            float W = 0.f, dW = 0.f;
            for (int k = 0; k < dim; ++k) A[k] = dA[k] = 0.f;
            for (int i = 0; i <= d; ++i) {
                const float bw = B[i] * w[i];
                W += bw;
                for (int k = 0; k < dim; ++k) A[k] = fmaf(bw, P[i][k], A[k]);
            }
            for (int i = 0; i < d; ++i) {
                const float bd = (float)d * Bd[i];
                dW = fmaf(bd, w[i + 1] - w[i], dW);
                for (int k = 0; k < dim; ++k) dA[k] = fmaf(bd, w[i + 1] * P[i + 1][k] - w[i] * P[i][k], dA[k]);
            }
            const float invW = 1.0f / W;
            float C[kGradMaxDim];
            for (int k = 0; k < dim; ++k) C[k] = A[k] * invW;
            for (int i = 0; i <= d; ++i) {
                const float f = B[i] * w[i] * invW;
                float dot = 0.f;
                for (int k = 0; k < dim; ++k) {
                    acc_c[i][k] = fmaf(f, gj[k], acc_c[i][k]);
                    dot = fmaf(P[i][k] - C[k], gj[k], dot);
                }
                acc_w[i] = fmaf(B[i] * invW, dot, acc_w[i]);
            }
            if (a.grad_t) {
                float gt = 0.f;
                for (int k = 0; k < dim; ++k) gt = fmaf(gj[k], fmaf(-C[k], dW, dA[k]), gt);
                gt = (traw >= 0.f && traw <= 1.f) ? gt * invW : 0.f;
                if (!shared_t) a.grad_t[c * a.n_t + j] = gt;
                else if (a.shared_gt) atomicAdd(s_gt + j, gt);
                else atomicAdd(a.grad_t + j, gt);
            }
        }
        // butterfly: every lane ends with the curve's sums; lane e writes element e
        const int nc = (d + 1) * dim;
        for (int i = 0; i <= d; ++i) {
            for (int k = 0; k < dim; ++k) {
                const float v = warp_sum(acc_c[i][k]);
                if (a.grad_ctrl && lane == (i * dim + k) % 32) a.grad_ctrl[c * nc + i * dim + k] = v;
            }
            const float vw = warp_sum(acc_w[i]);
            if (a.grad_w && lane == i % 32) a.grad_w[c * (d + 1) + i] = vw;
        }
    }
    if (shared_t && a.grad_t && a.shared_gt) {
        __syncthreads();
        for (int j = threadIdx.x; j < a.n_t; j += blockDim.x) atomicAdd(a.grad_t + j, s_gt[j]);
    }
}

LaunchResult launch_grad(const GradArgs& a, cudaStream_t s, const LaunchHooks& h)
{
    const void* kern;
    if (a.dim == 3) {
        switch (a.degree) {
        case 1: kern = (const void*)k_grad<1, 3>; break;
        case 2: kern = (const void*)k_grad<2, 3>; break;
        case 3: kern = (const void*)k_grad<3, 3>; break;
        case 4: kern = (const void*)k_grad<4, 3>; break;
        case 5: kern = (const void*)k_grad<5, 3>; break;
        case 6: kern = (const void*)k_grad<6, 3>; break;
        case 7: kern = (const void*)k_grad<7, 3>; break;
        default: kern = (const void*)k_grad<0, 3>; break;
        }
    } else {
        kern = (const void*)k_grad<0, 0>;
    }
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
