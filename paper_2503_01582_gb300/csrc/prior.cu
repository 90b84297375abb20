// Prior density grid support (§III-A "Normalized mesh generation", §III-B):
// the rays that query the field at the centres of an R^3 grid, and the yaw
// scores of the canonicalisation of Eq. 3.
#include <math.h>

#include <algorithm>

#include "device_common.cuh"

namespace prenom {

// One ray per (j, k) row of voxel centres: o = (0, (j+1/2)/R, (k+1/2)/R),
// d = (1, 0, 0), samples t_i = (i+1/2)/R -- the field at voxel (i, j, k) is
// then sample i of ray k R + j, x fastest.
__global__ void density_rays_kernel(int R, float *o, float *d, float *t)
{
    const int64_t n = (int64_t)R * R * R;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % R);
        const int64_t ray = q / R;
        t[q] = __fdiv_rn((float)i + 0.5f, (float)R);
        if (i == 0) {
            const int j = (int)(ray % R), k = (int)(ray / R);
            o[3 * ray] = 0.f;
            o[3 * ray + 1] = __fdiv_rn((float)j + 0.5f, (float)R);
            o[3 * ray + 2] = __fdiv_rn((float)k + 0.5f, (float)R);
            d[3 * ray] = 1.f;
            d[3 * ray + 1] = 0.f;
            d[3 * ray + 2] = 0.f;
        }
    }
}

constexpr int kYawThreads = 256;

// Deterministic block sum / min / max (fixed tree over the block's threads).
template <typename T, typename Op>
__device__ __forceinline__ T block_reduce(T v, T *sh, Op op)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kYawThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            sh[threadIdx.x] = op(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    const T r = sh[0];
    __syncthreads();
    return r;
}

// Block g scores yaw gamma_g = 2 pi g / n_gamma (Eq. 3): the cloud P (object
// frame, z up) turned about z, centred at the midpoint of its extents and
// divided by them (+1/2), and the prior density summed over its points
// (trilinear per point in FP32, the sum in FP64 in a fixed order).
__global__ void __launch_bounds__(kYawThreads) yaw_score_kernel(const float *grid, int R, const float *P, int n,
                                                                int n_gamma, double *score)
{
    __shared__ double shd[kYawThreads];
    __shared__ float shf[kYawThreads];
    const int g = blockIdx.x;
    const double gamma = 6.283185307179586476925286766559 * (double)g / (double)n_gamma;
    const float c = (float)cos(gamma), s = (float)sin(gamma);
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int j = threadIdx.x; j < n; j += kYawThreads) {
        const float x = P[3 * j], y = P[3 * j + 1], z = P[3 * j + 2];
        const float q[3] = {c * x - s * y, s * x + c * y, z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], q[a]);
            hi[a] = fmaxf(hi[a], q[a]);
        }
    }
    float mid[3], ext[3];
    bool flat[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float l = block_reduce(lo[a], shf, [](float u, float v) { return fminf(u, v); });
        const float h = block_reduce(hi[a], shf, [](float u, float v) { return fmaxf(u, v); });
        flat[a] = !(h > l);
        mid[a] = 0.5f * (l + h);
        ext[a] = h - l;
    }
    double acc = 0.0;
    for (int j = threadIdx.x; j < n; j += kYawThreads) {
        const float x = P[3 * j], y = P[3 * j + 1], z = P[3 * j + 2];
        const float q[3] = {c * x - s * y, s * x + c * y, z};
        float pn[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            pn[a] = flat[a] ? 0.5f : __fadd_rn(__fdiv_rn(q[a] - mid[a], ext[a]), 0.5f);
        acc += (double)prior_lookup(grid, R, pn[0], pn[1], pn[2]);
    }
    const double total = block_reduce(acc, shd, [](double u, double v) { return u + v; });
    if (threadIdx.x == 0)
        score[g] = total;
}

cudaError_t launch_density_rays(int R, float *o, float *d, float *t, cudaStream_t st)
{
    const int64_t n = (int64_t)R * R * R;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    density_rays_kernel<<<grid, 256, 0, st>>>(R, o, d, t);
    return cudaGetLastError();
}

cudaError_t launch_yaw_scores(const float *grid, int R, const float *P, int n, int n_gamma, double *score,
                              cudaStream_t st)
{
    yaw_score_kernel<<<n_gamma, kYawThreads, 0, st>>>(grid, R, P, n, n_gamma, score);
    return cudaGetLastError();
}

}  // namespace prenom
