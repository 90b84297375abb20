// Split execution of the training step.
//
// Inside the fused kernels (two 80 KB tensor-core CTAs, or one 176 KB FP32 CTA,
// per SM) the hash gathers of the encoding and the reductions of its adjoint
// are latency-bound: too few warps are in flight to cover L2 latency.  The
// split form runs them as kernels of their own at several times the occupancy
// and hands the tile data over through L2-sized buffers:
//   1. sample_encode_kernel: one warp per 1-4 rays: prior sampling (a1-a5) of
//      each, then the hash encoding (a6) of all their samples, one per lane;
//      writes each ray's data as the MLP kernel keeps it, the sample depths [ray][nr] and each tile's encoding as
//      the exact image the MLP kernel works on (16-bit: its tcgen05 A operand,
//      no-swizzle interleaved core matrices; FP32: feature-major rows);
//   2. fused_tc_kernel / fused_fp32_kernel in split mode: copy all three in,
//      run the MLP, compositing, loss and MLP backward (a7-a10) and write
//      dL/d(encoding) per tile, FP32, level-major, instead of scattering it;
//   3. hash_scatter_kernel: the hash-grid scatter (a10) of those gradients.
// The arithmetic of every step is the fused kernels' own code.  The hand-over
// buffers are written and read once with evict-first hints (st.cs / ld.cs), so
// that where they exceed L2 (a batched step of many objects) they do not evict
// the hash tables and gradient tables that the gathers and reductions reuse.
#pragma once

#include "fused_tc.cuh"

namespace prenom {

constexpr int kEncWarps = kThreads / 32;
constexpr int kEncMaxRays = 4;  // rays a warp samples before it encodes their samples together

// Rays per warp task of the sampling-encoding kernel: the fewest whose samples
// fill whole 32-lane rounds of the encoding loop (nr = 48: two rays, three full
// rounds instead of a full and a half-empty one), at most kEncMaxRays and
// kMaxNr samples.
__host__ __device__ __forceinline__ int enc_rays_per_warp(int nr)
{
    int r = 1;
    while ((r * nr) % 32 != 0 && 2 * r <= kEncMaxRays && 2 * r * nr <= kMaxNr)
        r *= 2;
    return r;
}

// FMT: 0 FP16 or 1 BF16 image in the tensor-core kernel's operand layout, 2 FP32
// feature-major image [IN][kSplitTile] for the FP32 kernel.
// F16: the items' gathers read the BF16 copies of their tables (FMT 0 or 1 only).
// MINB: resident CTAs per SM the registers are budgeted for (4: 64 registers a
// thread; 3: more registers and fewer warps, which suits gathers that hit in
// L1 and L2 better than gathers that go to DRAM; the autotuner picks per group).
template <int FMT, bool F16, int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
    sample_encode_kernel(const __grid_constant__ WorkItem one, const WorkList wl)
{
    using Hf = Half<FMT == 1>;
    __shared__ float s_rf[kEncWarps][kEncMaxRays][kRayStride];
    __shared__ float s_ts[kEncWarps][kMaxNr];
    __shared__ float s_cdf[kEncWarps][kMaxNc + 1];
    __shared__ int4 s_ray[kEncWarps][kEncMaxRays];  // (item, tile, row of the tile's first sample, ray) or item -1
    const WorkItem *list = wl.items ? wl.items : &one;
    const int n_items = wl.items ? wl.n_items : 1;
    const int total = wl.items ? wl.total_tiles : one.bd.n_tiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int NR = list[0].bd.rays_per_tile;  // the same for every item of a launch
    const int nr = list[0].bd.nr;             // likewise
    const int RW = enc_rays_per_warp(nr);
    const long long slots = (long long)total * NR;
    const long long tasks = (slots + RW - 1) / RW;
    float *ts = s_ts[warp];
    float *cdf = s_cdf[warp];
    // task q = warp * gridDim.x + block (+ multiples of the grid's warp count):
    // every block gets the same number of rays, to within RW, so the SMs share
    // the gathers evenly whatever the slot count
    for (long long q = (long long)warp * gridDim.x + blockIdx.x; q < tasks; q += (long long)gridDim.x * kEncWarps) {
        // 1. sampling, one ray after the other (each warp-wide)
        for (int r = 0; r < RW; ++r) {
            const long long j = q * RW + r;
            int4 meta = make_int4(-1, 0, 0, 0);
            if (j < slots) {
                const int t = (int)(j / NR), rr = (int)(j % NR);
                const int ii = item_of_tile(list, n_items, t);
                const WorkItem &it = list[ii];
                const int tile = t - it.tile_begin;
                const int gr = tile * NR + rr;
                if (gr < it.bd.n_rays) {  // else a slot past the batch's last ray (its rows stay unread)
                    meta = make_int4(ii, tile, rr * nr, gr);
                    float *rf = s_rf[warp][r];
                    if (lane < 4)
                        load_ray_fields(it.bd, gr, rf, lane);
                    __syncwarp();
                    sample_ray_warp(it.od, it.bd, r, gr, rf, ts, cdf, lane);  // also sets rf[RF_TN], rf[RF_TF]
                    __syncwarp();  // lane 0 wrote rf[RF_TN], rf[RF_TF]
                    if (lane < kRayStride)  // the ray's data for the tensor-core kernel
                        it.bd.sp_rays[((size_t)tile * kTcRayMax + rr) * kRayStride + lane] = rf[lane];
                    __syncwarp();  // cdf is rewritten by the next ray
                }
            }
            if (lane == 0)
                s_ray[warp][r] = meta;
        }
        __syncwarp();
        // 2. encoding of all samples of the task's rays, one per lane
        for (int s = lane; s < RW * nr; s += 32) {
            const int r = s / nr, k = s - r * nr;
            const int4 meta = s_ray[warp][r];
            if (meta.x < 0)
                continue;
            const WorkItem &it = list[meta.x];
            const ObjDesc &od = it.od;
            const BatchDesc &bd = it.bd;
            const float *rf = s_rf[warp][r];
            const int NL = od.IN / 2, INP = od.IN < 16 ? 16 : od.IN;
            const float2 *tab = reinterpret_cast<const float2 *>(od.theta);
            unsigned char *img = reinterpret_cast<unsigned char *>(bd.sp_x) + (size_t)meta.y * kSplitXBytes;
            const float tk = ts[s];
            bd.sp_t[(size_t)meta.w * nr + k] = tk;
            const float enc = (FMT != 2 && bd.enc_scale) ? *bd.enc_scale : 1.f;  // exact power of two
            float ph[3], pl[3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
                pos_two_float(rf[RF_O + a], tk, rf[RF_D + a], ph[a], pl[a]);
            const int row = meta.z + k;  // row of the tile image
            // levels in chunks of four, one 16-byte chunk of the row each (stored as soon as
            // it is complete); the chunk loop is not unrolled, which keeps the kernel's code
            // within the instruction cache (the unrolled 16-level body stalled its warps on
            // instruction fetch)
#pragma unroll 1
            for (int l4 = 0; l4 < kMaxLevels; l4 += 4) {
                if (l4 >= NL && (FMT == 2 || l4 / 4 >= INP / 8))
                    break;
                uint32_t pk[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int l = l4 + j;
                    pk[j] = 0u;
                    if (l < NL) {
                        const LevelDesc lv = od.lv[l];
                        Corners cs;
                        level_corners(lv, od.tmask, ph, pl, cs);
                        PRENOM_CHECK_CORNERS(lv, od.tmask, cs, bd.status);
                        float2 f[8];
                        if constexpr (F16) {  // the tables' BF16 copy
#pragma unroll
                            for (int c = 0; c < 8; c += 2)
                                gather_pair16(od.feat16 + lv.offset, cs.idx[c], cs.idx[c + 1], f[c], f[c + 1]);
                        } else {
#pragma unroll
                            for (int c = 0; c < 8; c += 2)
                                gather_pair(tab + lv.offset, cs.idx[c], cs.idx[c + 1], f[c], f[c + 1]);
                        }
                        float e0 = 0.f, e1 = 0.f;
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            e0 = fmaf(cs.wt[c], f[c].x, e0);
                            e1 = fmaf(cs.wt[c], f[c].y, e1);
                        }
                        if constexpr (FMT == 2) {  // consecutive lanes write consecutive samples of a feature
                            float *fimg = reinterpret_cast<float *>(img);
                            fimg[(2 * l) * kSplitTile + row] = e0;
                            fimg[(2 * l + 1) * kSplitTile + row] = e1;
                        } else {
                            pk[j] = Hf::pack2(e0 * enc, e1 * enc);
                        }
                    }
                }
                // row of the tile image: INP / 8 chunks of 8 columns (16 bytes each)
                if constexpr (FMT != 2) {
                    if (l4 / 4 < INP / 8)
                        __stcs(reinterpret_cast<uint4 *>(img + il_off(row, 2 * l4, INP)),
                               make_uint4(pk[0], pk[1], pk[2], pk[3]));
                }
            }
        }
        __syncwarp();  // s_rf, s_ts and s_ray are rewritten by the next task
    }
}

template <int FMT>
cudaError_t launch_sample_encode_t(const WorkItem &one, const WorkList &wl, int per_sm, int grid, cudaStream_t st)
{
    if constexpr (FMT != 2) {
        if (wl.feat16) {
            if (per_sm == 3)
                sample_encode_kernel<FMT, true, 3><<<grid, kThreads, 0, st>>>(one, wl);
            else
                sample_encode_kernel<FMT, true, 4><<<grid, kThreads, 0, st>>>(one, wl);
            return cudaGetLastError();
        }
    }
    if (per_sm == 3)
        sample_encode_kernel<FMT, false, 3><<<grid, kThreads, 0, st>>>(one, wl);
    else
        sample_encode_kernel<FMT, false, 4><<<grid, kThreads, 0, st>>>(one, wl);
    return cudaGetLastError();
}

}  // namespace prenom
