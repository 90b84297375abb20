// The fused FP32 training kernel and its launchers (device stages in fused_fp32.cuh).
//
// A launch runs a work list: one or many (object, ray batch) items whose MLP
// width W and encoding width IN match; the items' tiles are numbered across
// the list and each persistent CTA walks one contiguous range of them.  When
// the range crosses into another object the CTA flushes its weight-gradient
// accumulators and loss into the previous object and loads the next one's
// weights, so dozens of objects of different table sizes, depths and ray
// counts share one launch.
#pragma once

#include "fused_fp32.cuh"

namespace prenom {

// Weights of one object into shared memory: Wb = theta layout [out][in],
// Wf = per-layer transpose [in][out]; gradient accumulators cleared.
template <int W, int IN>
__device__ __forceinline__ void fp32_load_object(const ObjDesc &od, float *Wf, float *Wb, float *dWs)
{
    const int H = od.H;
    const int nW = IN * W + (H - 1) * W * W + 4 * W;
    const int off_out = IN * W + (H - 1) * W * W;
    const float *th = od.theta + od.mlp_off;
    for (int i = threadIdx.x; i < nW; i += kThreads) {
        const float v = th[i];
        Wb[i] = v;
        dWs[i] = 0.f;
        int lo, nin, nout, j;
        if (i < IN * W) {
            lo = 0; nin = IN; nout = W; j = i;
        } else if (i < off_out) {
            const int jj = i - IN * W;
            lo = IN * W + (jj / (W * W)) * W * W; nin = W; nout = W; j = jj % (W * W);
        } else {
            lo = off_out; nin = W; nout = 4; j = i - off_out;
        }
        Wf[lo + (j % nin) * nout + (j / nin)] = v;
    }
    __syncthreads();
}

// Accumulated loss and weight gradients of the CTA into the object.
template <int W, int IN>
__device__ __forceinline__ void fp32_flush_object(const ObjDesc &od, const BatchDesc &bd, float *dWs, float &loss_acc)
{
    if ((threadIdx.x & 31) == 0 && bd.mode == kTrain && loss_acc != 0.f)
        red_add_f(bd.loss, loss_acc);
    loss_acc = 0.f;
    if (bd.mode != kRender) {
        // nW is a multiple of 4 and the MLP block is 16-byte aligned (the hash levels are
        // padded to 8 two-feature entries): 16-byte reductions, a quarter of the requests
        const int nW = IN * W + (od.H - 1) * W * W + 4 * W;
        float4 *gw = reinterpret_cast<float4 *>(od.grad + od.mlp_off);
        const float4 *src = reinterpret_cast<const float4 *>(dWs);
        for (int i = threadIdx.x; i < nW / 4; i += kThreads) {
            const float4 v = src[i];
            if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)
                red_add_f4(gw + i, v.x, v.y, v.z, v.w);
        }
    }
    __syncthreads();
}

template <int W, int IN, int S>
__global__ void __launch_bounds__(kThreads, 1)
    fused_fp32_kernel(const __grid_constant__ WorkItem one, const WorkList wl)
{
    constexpr int SP = S + 4;
    constexpr int MAXR = S / kMinNr;
    extern __shared__ __align__(16) float sm[];
    const WorkItem *list = wl.items ? wl.items : &one;
    const int n_items = wl.items ? wl.n_items : 1;
    const int total = wl.items ? wl.total_tiles : one.bd.n_tiles;
    const int hmax = wl.items ? wl.hmax : one.od.H;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nWmax = IN * W + (hmax - 1) * W * W + 4 * W;  // multiple of 4
    float *Wf = sm;               // [in][out] per layer (forward operand)
    float *Wb = Wf + nWmax;       // [out][in] per layer (backward operand, = theta layout)
    float *dWs = Wb + nWmax;      // weight-gradient accumulators, [out][in]
    float *XT = dWs + nWmax;      // [IN][SP]: encoding, then dL/dX
    float *HT = XT + IN * SP;     // [H][W][SP]: activations, then dL/dH in place
    float *OT = HT + hmax * W * SP;  // [4][SP] raw outputs
    float *dOT = OT + 4 * SP;     // [4][SP] dL/d(raw outputs)
    float *ts = dOT + 4 * SP;     // [SP] sample depths
    float *rayf = ts + SP;        // [MAXR][16]
    float *cdfs = rayf + MAXR * kRayStride;  // [8][kMaxNc + 1]

    __shared__ __align__(16) WorkItem cur;  // the item being processed
    const int per = (total + (int)gridDim.x - 1) / (int)gridDim.x;
    const int t0 = (int)blockIdx.x * per, t1 = min(total, t0 + per);
    int k = -1;
    float loss_acc = 0.f;
    for (int t = t0; t < t1; ++t) {
        int nk = k < 0 ? item_of_tile(list, n_items, t) : k;
        while (nk + 1 < n_items && list[nk + 1].tile_begin <= t)
            ++nk;
        if (nk != k) {
            if (k >= 0)
                fp32_flush_object<W, IN>(cur.od, cur.bd, dWs, loss_acc);
            stage_item(list[nk], cur);
            fp32_load_object<W, IN>(cur.od, Wf, Wb, dWs);
            k = nk;
        }
        const ObjDesc &od = cur.od;
        const BatchDesc &bd = cur.bd;
        const int H = od.H;
        const int off_out = IN * W + (H - 1) * W * W;
        const int nr = bd.nr, NR = bd.rays_per_tile;
        const int tile = t - cur.tile_begin;
        const int ray0 = tile * NR;
        const int nrt = min(NR, bd.n_rays - ray0);
        const int ns = nrt * nr;
        const bool split = bd.sp_x != nullptr;  // sampling, encoding and scatter run in kernels of their own
        if (split) {
            // (1-3) the tile's ray data, sample depths and FP32 encoding from the
            // sampling-encoding kernel (rows past the tile's samples zeroed)
            const float *rsrc = bd.sp_rays + (size_t)tile * kSplitRayFloats;
            for (int i = tid; i < nrt * kRayStride; i += kThreads)
                rayf[i] = rsrc[i];
            for (int i = tid; i < ns; i += kThreads)
                ts[i] = bd.sp_t[(size_t)ray0 * nr + i];
            const float *img = reinterpret_cast<const float *>(bd.sp_x) + (size_t)tile * (kSplitXBytes / 4);
            for (int i = tid; i < IN * S; i += kThreads) {
                const int c = i / S, s = i % S;
                XT[c * SP + s] = s < ns ? img[c * kSplitTile + s] : 0.f;
            }
            if (tid < S && tid >= ns)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    dOT[c * SP + tid] = 0.f;
            __syncthreads();
        } else {
            // (1) ray data
            load_ray_tile(bd, ray0, nrt, rayf);
            __syncthreads();
            // (2) sampling
            for (int r = warp; r < nrt; r += kThreads / 32)
                sample_ray_warp(od, bd, r, ray0 + r, rayf + r * kRayStride, ts, cdfs + warp * (kMaxNc + 1), lane);
            __syncthreads();
            // (3) encoding
            encode_or_scatter<IN, S, false>(od, bd, rayf, ts, XT, dOT, ns);
            __syncthreads();
        }
        // (4) MLP forward
        gemm_sn<S, W, kRelu>(XT, Wf, IN, HT);
        __syncthreads();
        for (int l = 1; l < H; ++l) {
            gemm_sn<S, W, kRelu>(HT + (l - 1) * W * SP, Wf + IN * W + (l - 1) * W * W, W, HT + l * W * SP);
            __syncthreads();
        }
        out_layer_fwd<W, S>(HT + (H - 1) * W * SP, Wf + off_out, OT);
        __syncthreads();
        // (5) compositing, loss and its adjoint
        // (the sampler's CDF scratch serves as the compositing's exchange buffer)
        loss_acc += composite_tile(od, bd, ray0, nrt, rayf, ts, OT, dOT, SP, cdfs);
        __syncthreads();
        if (bd.mode == kRender)
            continue;
        // (6) MLP backward
        gemm_dw<S, 4, W>(dOT, HT + (H - 1) * W * SP, dWs + off_out);
        __syncthreads();
        gemm_sn<S, W, kMaskByOld>(dOT, Wb + off_out, 4, HT + (H - 1) * W * SP);
        __syncthreads();
        for (int l = H - 1; l >= 1; --l) {
            gemm_dw<S, W, W>(HT + l * W * SP, HT + (l - 1) * W * SP, dWs + IN * W + (l - 1) * W * W);
            __syncthreads();
            gemm_sn<S, W, kMaskByOld>(HT + l * W * SP, Wb + IN * W + (l - 1) * W * W, W, HT + (l - 1) * W * SP);
            __syncthreads();
        }
        gemm_dw<S, W, IN>(HT, XT, dWs);
        __syncthreads();
        gemm_sn<S, IN, kStore>(HT, Wb, W, XT);
        __syncthreads();
        // (7) hash-grid scatter, or dL/d(encoding) to the scatter kernel (level-major pairs)
        if (split) {
            float2 *dx = bd.sp_dx + (size_t)tile * kSplitDx;
            for (int i = tid; i < (IN / 2) * S; i += kThreads) {
                const int l = i / S, s = i % S;
                if (s < ns)
                    dx[l * kSplitTile + s] = make_float2(XT[(2 * l) * SP + s], XT[(2 * l + 1) * SP + s]);
            }
        } else {
            encode_or_scatter<IN, S, true>(od, bd, rayf, ts, XT, dOT, ns);
        }
        __syncthreads();
    }
    if (k >= 0)
        fp32_flush_object<W, IN>(cur.od, cur.bd, dWs, loss_acc);
}

inline size_t fused_fp32_smem_floats(int W, int IN, int H, int S)
{
    const size_t SP = (size_t)S + 4;
    const size_t nW = (size_t)IN * W + (size_t)(H - 1) * W * W + 4 * (size_t)W;
    return 3 * nW + IN * SP + (size_t)H * W * SP + 8 * SP + SP + (size_t)(S / kMinNr) * kRayStride +
           8 * (size_t)(kMaxNc + 1);
}

template <int W, int IN, int S>
cudaError_t launch_fused_t(const WorkItem &one, const WorkList &wl, int grid, cudaStream_t st)
{
    const int hmax = wl.items ? wl.hmax : one.od.H;
    const size_t smem = fused_fp32_smem_floats(W, IN, hmax, S) * sizeof(float);
    cudaError_t e = allow_max_dynamic_smem(fused_fp32_kernel<W, IN, S>);
    if (e != cudaSuccess)
        return e;
    fused_fp32_kernel<W, IN, S><<<grid, kThreads, smem, st>>>(one, wl);
    return cudaGetLastError();
}

template <int W>
cudaError_t launch_fused_w(const WorkItem &one, const WorkList &wl, int IN, int S, int grid, cudaStream_t st)
{
    if (S == 128) {
        switch (IN) {
        case 8: return launch_fused_t<W, 8, 128>(one, wl, grid, st);
        case 16: return launch_fused_t<W, 16, 128>(one, wl, grid, st);
        case 32: return launch_fused_t<W, 32, 128>(one, wl, grid, st);
        default: return cudaErrorInvalidValue;
        }
    }
    if constexpr (W == 64) {  // only the widest MLP ever needs the smaller tile
        if (S != 64)
            return cudaErrorInvalidValue;
        switch (IN) {
        case 8: return launch_fused_t<W, 8, 64>(one, wl, grid, st);
        case 16: return launch_fused_t<W, 16, 64>(one, wl, grid, st);
        case 32: return launch_fused_t<W, 32, 64>(one, wl, grid, st);
        default: return cudaErrorInvalidValue;
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace prenom
