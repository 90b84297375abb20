// Meta-learning kernels (§III-A): the start of a Reptile meta step (every task
// object receives the meta-parameters and fresh Adam state) and the outer
// update of Eq. 2 over a meta-batch of tasks, theta <- theta + beta (mean_t
// theta_t - theta).  Arrays are 16-byte aligned; the first n/4 quadruples are
// float4 accesses and the remaining n % 4 elements scalar ones.
#include "prenom_internal.h"

namespace prenom {

__device__ __forceinline__ float reptile_step(float th, float s, float beta, float nf)
{
    return th + beta * (__fdiv_rn(s, nf) - th);
}

__global__ void reptile_broadcast_kernel(const ReptileArgs a)
{
    const int64_t n4 = a.n / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 th = reinterpret_cast<const float4 *>(a.meta)[i];
        for (int t = 0; t < a.n_tasks; ++t) {
            reinterpret_cast<float4 *>(a.theta[t])[i] = th;
            // gradient, Adam m and v follow theta in the task's arena, n_pad apart
            reinterpret_cast<float4 *>(a.theta[t] + a.n_pad)[i] = z;
            reinterpret_cast<float4 *>(a.theta[t] + 2 * a.n_pad)[i] = z;
            reinterpret_cast<float4 *>(a.theta[t] + 3 * a.n_pad)[i] = z;
        }
    }
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
        for (int t = 0; t < a.n_tasks; ++t) {
            a.theta[t][i] = a.meta[i];
            a.theta[t][a.n_pad + i] = 0.f;
            a.theta[t][2 * a.n_pad + i] = 0.f;
            a.theta[t][3 * a.n_pad + i] = 0.f;
        }
}

// Sum of the tasks' parameters in task order; with a.meta set the outer update
// is applied directly (single GPU), otherwise the sum goes to a.sum (the ranks
// of a multi-GPU meta step add their sums before reptile_apply_kernel).
__global__ void reptile_sum_kernel(const ReptileArgs a)
{
    const int64_t n4 = a.n / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        float4 s = reinterpret_cast<const float4 *>(a.theta[0])[i];
        for (int t = 1; t < a.n_tasks; ++t) {
            const float4 v = reinterpret_cast<const float4 *>(a.theta[t])[i];
            s.x += v.x;
            s.y += v.y;
            s.z += v.z;
            s.w += v.w;
        }
        if (a.meta) {
            float4 th = reinterpret_cast<float4 *>(a.meta)[i];
            th.x = reptile_step(th.x, s.x, a.beta, a.nf);
            th.y = reptile_step(th.y, s.y, a.beta, a.nf);
            th.z = reptile_step(th.z, s.z, a.beta, a.nf);
            th.w = reptile_step(th.w, s.w, a.beta, a.nf);
            reinterpret_cast<float4 *>(a.meta)[i] = th;
        } else {
            reinterpret_cast<float4 *>(a.sum)[i] = s;
        }
    }
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        float s = a.theta[0][i];
        for (int t = 1; t < a.n_tasks; ++t)
            s += a.theta[t][i];
        if (a.meta)
            a.meta[i] = reptile_step(a.meta[i], s, a.beta, a.nf);
        else
            a.sum[i] = s;
    }
}

__global__ void reptile_apply_kernel(const ReptileArgs a)
{
    const int64_t n4 = a.n / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 s = reinterpret_cast<const float4 *>(a.sum)[i];
        float4 th = reinterpret_cast<float4 *>(a.meta)[i];
        th.x = reptile_step(th.x, s.x, a.beta, a.nf);
        th.y = reptile_step(th.y, s.y, a.beta, a.nf);
        th.z = reptile_step(th.z, s.z, a.beta, a.nf);
        th.w = reptile_step(th.w, s.w, a.beta, a.nf);
        reinterpret_cast<float4 *>(a.meta)[i] = th;
    }
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
        a.meta[i] = reptile_step(a.meta[i], a.sum[i], a.beta, a.nf);
}

cudaError_t launch_reptile(const ReptileArgs &a, int op, int grid, cudaStream_t st)
{
    switch (op) {
    case kReptileBroadcast: reptile_broadcast_kernel<<<grid, 256, 0, st>>>(a); break;
    case kReptileSum: reptile_sum_kernel<<<grid, 256, 0, st>>>(a); break;
    case kReptileApply: reptile_apply_kernel<<<grid, 256, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace prenom
