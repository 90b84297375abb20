// Split execution of the training step.
//
// Inside the fused kernels (two 80 KB tensor-core CTAs, or one 176 KB FP32 CTA,
// per SM) the hash gathers of the encoding and the reductions of its adjoint
// are latency-bound: too few warps are in flight to cover L2 latency.  The
// split form runs them as kernels of their own at several times the occupancy
// and hands the tile data over through L2-sized buffers:
//   1. sample_encode_kernel: one warp per ray: prior sampling (a1-a5) and the
//      hash encoding (a6) of its samples; writes each ray's data as the MLP
//      kernel keeps it, the sample depths [ray][nr] and each tile's encoding as
//      the exact image the MLP kernel works on (16-bit: its tcgen05 A operand,
//      no-swizzle interleaved core matrices; FP32: feature-major rows);
//   2. fused_tc_kernel / fused_fp32_kernel in split mode: copy all three in,
//      run the MLP, compositing, loss and MLP backward (a7-a10) and write
//      dL/d(encoding) per tile, FP32, level-major, instead of scattering it;
//   3. hash_scatter_kernel: the hash-grid scatter (a10) of those gradients.
// The arithmetic of every step is the fused kernels' own code.
#pragma once

#include "fused_tc.cuh"

namespace prenom {

constexpr int kEncWarps = kThreads / 32;

// FMT: 0 FP16 or 1 BF16 image in the tensor-core kernel's operand layout, 2 FP32
// feature-major image [IN][kSplitTile] for the FP32 kernel.
template <int FMT>
__global__ void __launch_bounds__(kThreads, 4)
    sample_encode_kernel(const __grid_constant__ WorkItem one, const WorkList wl)
{
    using Hf = Half<FMT == 1>;
    __shared__ float s_rf[kEncWarps][kRayStride];
    __shared__ float s_ts[kEncWarps][kMaxNr];
    __shared__ float s_cdf[kEncWarps][kMaxNc + 1];
    const WorkItem *list = wl.items ? wl.items : &one;
    const int n_items = wl.items ? wl.n_items : 1;
    const int total = wl.items ? wl.total_tiles : one.bd.n_tiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int NR = list[0].bd.rays_per_tile;  // the same for every item of a launch
    const long long slots = (long long)total * NR;
    float *rf = s_rf[warp];
    float *ts = s_ts[warp];
    float *cdf = s_cdf[warp];
    // ray slot j = warp * gridDim.x + block (+ multiples of the grid's warp count):
    // every block gets the same number of rays, to within one, so the SMs share
    // the gathers evenly whatever the slot count
    for (long long j = (long long)warp * gridDim.x + blockIdx.x; j < slots; j += (long long)gridDim.x * kEncWarps) {
        const int t = (int)(j / NR), rr = (int)(j % NR);
        const WorkItem &it = list[item_of_tile(list, n_items, t)];
        const ObjDesc &od = it.od;
        const BatchDesc &bd = it.bd;
        const int tile = t - it.tile_begin;
        const int gr = tile * NR + rr;
        if (gr >= bd.n_rays)  // ray slot past the batch's last ray (the tile's rows stay unread)
            continue;
        if (lane < 4)
            load_ray_fields(bd, gr, rf, lane);
        __syncwarp();
        sample_ray_warp(od, bd, 0, gr, rf, ts, cdf, lane);  // also sets rf[RF_TN], rf[RF_TF]
        if (lane < kRayStride)  // the ray's data for the tensor-core kernel
            bd.sp_rays[((size_t)tile * kTcRayMax + rr) * kRayStride + lane] = rf[lane];
        const int nr = bd.nr, NL = od.IN / 2, INP = od.IN < 16 ? 16 : od.IN;
        const float2 *tab = reinterpret_cast<const float2 *>(od.theta);
        unsigned char *img = reinterpret_cast<unsigned char *>(bd.sp_x) + (size_t)tile * kSplitXBytes;
        for (int k = lane; k < nr; k += 32) {
            const float tk = ts[k];
            bd.sp_t[(size_t)gr * nr + k] = tk;
            float ph[3], pl[3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                pos_two_float(rf[RF_O + a], tk, rf[RF_D + a], ph[a], pl[a]);
            const int s = rr * nr + k;  // row of the tile image
            uint32_t pk[4];  // one 16-byte chunk (4 levels) of the row, stored as soon as it is complete
#pragma unroll
            for (int l = 0; l < kMaxLevels; ++l) {
                pk[l & 3] = 0u;
                if (l < NL) {
                    const LevelDesc lv = od.lv[l];
                    Corners cs;
                    level_corners(lv, od.tmask, ph, pl, cs);
                    float2 f[8];
#pragma unroll
                    for (int c = 0; c < 8; c += 2)
                        gather_pair(tab + lv.offset, cs.idx[c], cs.idx[c + 1], f[c], f[c + 1]);
                    float e0 = 0.f, e1 = 0.f;
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        e0 = fmaf(cs.wt[c], f[c].x, e0);
                        e1 = fmaf(cs.wt[c], f[c].y, e1);
                    }
                    if constexpr (FMT == 2) {  // consecutive lanes write consecutive samples of a feature
                        float *fimg = reinterpret_cast<float *>(img);
                        fimg[(2 * l) * kSplitTile + s] = e0;
                        fimg[(2 * l + 1) * kSplitTile + s] = e1;
                    } else {
                        pk[l & 3] = (uint32_t)Hf::bits(e0) | ((uint32_t)Hf::bits(e1) << 16);
                    }
                }
                // row s of the tile image: INP / 8 chunks of 8 columns (16 bytes each)
                if constexpr (FMT != 2) {
                    if ((l & 3) == 3 && l / 4 < INP / 8)
                        *reinterpret_cast<uint4 *>(img + il_off(s, 8 * (l / 4), INP)) =
                            make_uint4(pk[0], pk[1], pk[2], pk[3]);
                }
            }
        }
        __syncwarp();  // rf and ts are rewritten for the next ray
    }
}

template <int FMT>
cudaError_t launch_sample_encode_t(const WorkItem &one, const WorkList &wl, int grid, cudaStream_t st)
{
    sample_encode_kernel<FMT><<<grid, kThreads, 0, st>>>(one, wl);
    return cudaGetLastError();
}

}  // namespace prenom
