// Hash-grid scatter kernel of the split training step, and the launchers of
// the split form's two extra kernels (the FP32 encoder is instantiated here).
#include "split_tc.cuh"

namespace prenom {

// The hash scatter of a work list from its dL/d(encoding) buffers.  Blocks walk
// contiguous tile ranges; a tile's sample positions are staged in shared
// memory once and each warp scatters one (level, 32 consecutive samples) at a
// time, so a warp's lanes hold neighbouring samples of one level.
__global__ void __launch_bounds__(kThreads, 5)
    hash_scatter_kernel(const __grid_constant__ WorkItem one, const WorkList wl)
{
    __shared__ __align__(16) WorkItem cur;
    __shared__ float s_p[6][kSplitTile];  // hi[3], lo[3] of each sample's position
    const WorkItem *list = wl.items ? wl.items : &one;
    const int n_items = wl.items ? wl.n_items : 1;
    const int total = wl.items ? wl.total_tiles : one.bd.n_tiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // contiguous tile ranges whose lengths differ by at most one
    const int t0 = (int)((long long)blockIdx.x * total / gridDim.x);
    const int t1 = (int)((long long)(blockIdx.x + 1) * total / gridDim.x);
    int k = -1;
    for (int t = t0; t < t1; ++t) {
        int nk = k < 0 ? item_of_tile(list, n_items, t) : k;
        while (nk + 1 < n_items && list[nk + 1].tile_begin <= t)
            ++nk;
        if (nk != k) {
            __syncthreads();
            stage_item(list[nk], cur);
            k = nk;
        }
        const ObjDesc &od = cur.od;
        const BatchDesc &bd = cur.bd;
        const int nr = bd.nr, NR = bd.rays_per_tile;
        const int tile = t - cur.tile_begin, ray0 = tile * NR;
        const int ns = min(NR, bd.n_rays - ray0) * nr;
        if ((int)threadIdx.x < ns) {
            const int s = threadIdx.x, gr = ray0 + s / nr;
            const float tk = bd.sp_t[(size_t)gr * nr + s % nr];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float hi, lo;
                pos_two_float(bd.o[(size_t)gr * 3 + a], tk, bd.d[(size_t)gr * 3 + a], hi, lo);
                s_p[a][s] = hi;
                s_p[3 + a][s] = lo;
            }
        }
        __syncthreads();
        const int NL = od.IN / 2;
        const float2 *dx = bd.sp_dx + (size_t)tile * kSplitDx;
        float2 *gtab = reinterpret_cast<float2 *>(od.grad);
        for (int task = warp; task < NL * (kSplitTile / 32); task += kEncWarps) {
            const int l = task / (kSplitTile / 32), c = task % (kSplitTile / 32);
            if (c * 32 >= ns)
                continue;  // warp-uniform
            const int s = c * 32 + lane;
            const bool active = s < ns;
            float ph[3], pl[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                ph[a] = active ? s_p[a][s] : 0.f;
                pl[a] = active ? s_p[3 + a][s] : 0.f;
            }
            const LevelDesc lv = od.lv[l];
            Corners cs;
            level_corners(lv, od.tmask, ph, pl, cs);
            const float2 g = active ? dx[l * kSplitTile + s] : make_float2(0.f, 0.f);
            scatter_level_warp(gtab + lv.offset, active, cs, g.x, g.y, lane);
        }
        __syncthreads();  // s_p is rewritten for the next tile
    }
}

cudaError_t launch_sample_encode_fp16(const WorkItem &one, const WorkList &wl, int grid, cudaStream_t st);
cudaError_t launch_sample_encode_bf16(const WorkItem &one, const WorkList &wl, int grid, cudaStream_t st);

cudaError_t launch_sample_encode(const WorkItem &one, const WorkList &wl, int precision, int grid, cudaStream_t st)
{
    if (precision == 0)
        return launch_sample_encode_t<2>(one, wl, grid, st);
    return precision == 2 ? launch_sample_encode_bf16(one, wl, grid, st) : launch_sample_encode_fp16(one, wl, grid, st);
}

cudaError_t launch_hash_scatter(const WorkItem &one, const WorkList &wl, int grid, cudaStream_t st)
{
    hash_scatter_kernel<<<grid, kThreads, 0, st>>>(one, wl);
    return cudaGetLastError();
}

}  // namespace prenom
