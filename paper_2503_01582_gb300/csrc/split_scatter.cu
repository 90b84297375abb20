// Hash-grid scatter kernel of the split training step, and the launchers of
// the split form's two extra kernels (the FP32 encoder is instantiated here).
#include "split_tc.cuh"

namespace prenom {

// The hash scatter of a work list from its dL/d(encoding) buffers.  Blocks
// take tiles round-robin (tile t goes to block t mod grid), so the tiles in
// flight at any moment are a window of about one grid's worth of consecutive
// tiles: one or two objects of a batched step, whose gradient tables then stay
// in L2 while their reductions land (with contiguous ranges per block every
// object of a group is in flight at once, and the tables of a group of larger
// objects miss L2 on every reduction).  A tile's sample positions are staged in
// shared memory, double-buffered with the tile's work item, so one block
// barrier per tile suffices; each warp then scatters one (level, 32 consecutive
// samples) at a time, so a warp's lanes hold neighbouring samples of one level.
// CHUNK_LOG2: lanes of one cell summed in chunks of 2^CHUNK_LOG2 (5: whole runs).
template <int CHUNK_LOG2>
__global__ void __launch_bounds__(kThreads, 5)
    hash_scatter_kernel(const __grid_constant__ WorkItem one, const WorkList wl)
{
    __shared__ __align__(16) WorkItem cur[2];
    __shared__ float s_p[2][6][kSplitTile];  // hi[3], lo[3] of each sample's position
    const WorkItem *list = wl.items ? wl.items : &one;
    const int n_items = wl.items ? wl.n_items : 1;
    const int total = wl.items ? wl.total_tiles : one.bd.n_tiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int held[2] = {-1, -1};  // item held in cur[0], cur[1] (block-uniform)
    int i = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x, ++i) {
        const int b = i & 1;  // readers of cur[b] and s_p[b] from two tiles ago passed the last barrier
        const int nk = item_of_tile(list, n_items, t);
        if (nk != held[b]) {
            const int *src = reinterpret_cast<const int *>(&list[nk]);
            int *dst = reinterpret_cast<int *>(&cur[b]);
            for (int q = threadIdx.x; q < (int)(sizeof(WorkItem) / sizeof(int)); q += kThreads)
                dst[q] = src[q];
            held[b] = nk;
        }
        const BatchDesc &gb = list[nk].bd;  // read directly until the barrier publishes cur[b]
        const int nr = gb.nr, NR = gb.rays_per_tile;
        const int tile = t - list[nk].tile_begin, ray0 = tile * NR;
        const int ns = min(NR, gb.n_rays - ray0) * nr;
        if ((int)threadIdx.x < ns) {
            const int s = threadIdx.x, gr = ray0 + s / nr;
            const float tk = gb.sp_t[(size_t)gr * nr + s % nr];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                float hi, lo;
                pos_two_float(gb.o[(size_t)gr * 3 + a], tk, gb.d[(size_t)gr * 3 + a], hi, lo);
                s_p[b][a][s] = hi;
                s_p[b][3 + a][s] = lo;
            }
        }
        __syncthreads();
        const ObjDesc &od = cur[b].od;
        const BatchDesc &bd = cur[b].bd;
        const int NL = od.IN / 2;
        const float2 *dx = bd.sp_dx + (size_t)tile * kSplitDx;
        float2 *gtab = reinterpret_cast<float2 *>(od.grad);
        // the tile's (level, 32-sample chunk) tasks, over the filled chunks only, dealt
        // round-robin to the warps (skipping empty chunks instead left whole warps idle
        // at the barrier: a tile of two 48-sample rays fills 3 of 4 chunks)
        const int nch = (ns + 31) >> 5;
        for (int task = warp; task < NL * nch; task += kEncWarps) {
            const int l = task / nch, c = task - l * nch;
            const int s = c * 32 + lane;
            const bool active = s < ns;
            float ph[3], pl[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                ph[a] = active ? s_p[b][a][s] : 0.f;
                pl[a] = active ? s_p[b][3 + a][s] : 0.f;
            }
            const LevelDesc lv = od.lv[l];
            Corners cs;
            level_corners(lv, od.tmask, ph, pl, cs);
            PRENOM_CHECK_CORNERS(lv, od.tmask, cs, bd.status);
            const float2 g = active ? __ldcs(dx + l * kSplitTile + s) : make_float2(0.f, 0.f);  // read once
            scatter_level_warp<CHUNK_LOG2>(gtab + lv.offset, active, cs, g.x, g.y, lane);
        }
    }
}

cudaError_t launch_sample_encode_fp16(const WorkItem &one, const WorkList &wl, int per_sm, int grid, cudaStream_t st);
cudaError_t launch_sample_encode_bf16(const WorkItem &one, const WorkList &wl, int per_sm, int grid, cudaStream_t st);

cudaError_t launch_sample_encode(const WorkItem &one, const WorkList &wl, int precision, int per_sm, int grid,
                                 cudaStream_t st)
{
    if (precision == 0)
        return launch_sample_encode_t<2>(one, wl, per_sm, grid, st);
    return precision == 2 ? launch_sample_encode_bf16(one, wl, per_sm, grid, st)
                          : launch_sample_encode_fp16(one, wl, per_sm, grid, st);
}

cudaError_t launch_hash_scatter(const WorkItem &one, const WorkList &wl, int grid, cudaStream_t st, bool whole_runs)
{
    if (whole_runs)
        hash_scatter_kernel<5><<<grid, kThreads, 0, st>>>(one, wl);
    else
        hash_scatter_kernel<kScatterChunkLog2><<<grid, kThreads, 0, st>>>(one, wl);
    return cudaGetLastError();
}

}  // namespace prenom
