// Adam update over every parameter of a step's objects, random initialisation,
// and the host-side dispatch of the fused kernels.
#include "fused_fp32_kernel.cuh"
#include "fused_tc.cuh"

namespace prenom {

// ---------------------------------------------------------------- Adam
// Dense Adam (Kingma & Ba) with bias correction, streamed once over theta,
// grad, m and v of all segments (32 bytes moved per parameter: 16 read, 16
// written, the gradient being zeroed for the next step's atomics).  Work is
// cut into 1024-float chunks numbered across segments (4096-float chunks left
// a tail of a few long chunks: 63.1 against 59.5 us on a 12.2 M-parameter
// object); a block finds its segment by binary search over the chunk prefix
// sums held in parameter space.
__device__ __forceinline__ void adam_one(float &th, float &m, float &v, float g, float b1, float b2, float eps,
                                         float lr_c1, float inv_c2)
{
    m = fmaf(b1, m, (1.f - b1) * g);
    v = fmaf(b2, v, (1.f - b2) * g * g);
    th -= lr_c1 * m / (sqrtf(v * inv_c2) + eps);
}

// Two FP32 values as one bf16x2 word, the first in the low half (rounded to nearest even).
__device__ __forceinline__ uint32_t bf16_pair(float a, float b)
{
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}

// max |x| of a warp into *dst (non-negative floats order like their bit patterns)
__device__ __forceinline__ void warp_absmax_to(uint32_t *dst, float amax)
{
    const uint32_t m = __reduce_max_sync(kFull, __float_as_uint(amax));
    if ((threadIdx.x & 31) == 0 && m != 0u)
        atomicMax(dst, m);
}

__global__ void __launch_bounds__(256) adam_kernel(const AdamArgs a)
{
    const int64_t total = a.chunk_start[a.n_segs];
    int cur = -1;       // segment whose updated hash entries amax covers (block-uniform)
    float amax = 0.f;   // this thread's max |theta| over them
    bool skip = false;  // the current segment's step is dropped
    float lr_c1 = 0.f, inv_c2 = 0.f;
    for (int64_t c = blockIdx.x; c < total; c += gridDim.x) {
        int lo = 0, hi = a.n_segs - 1;
        while (lo < hi) {  // last segment whose first chunk is <= c
            const int mid = (lo + hi + 1) >> 1;
            if (a.chunk_start[mid] <= c)
                lo = mid;
            else
                hi = mid - 1;
        }
        const AdamSeg &sg = a.seg[lo];
        if (lo != cur) {  // the segment's flag and factors, read once per segment, not once per chunk
            if (cur >= 0 && a.seg[cur].absmax)
                warp_absmax_to(a.seg[cur].absmax, amax);
            cur = lo;
            amax = 0.f;
            skip = sg.skip && *sg.skip;
            lr_c1 = sg.lr_c1;
            inv_c2 = sg.inv_c2;
            if (sg.scal) {
                const float2 s = *sg.scal;
                lr_c1 = s.x;
                inv_c2 = s.y;
            }
        }
        const int64_t base = (c - a.chunk_start[lo]) * kAdamChunk;
        const int64_t end = min(base + (int64_t)kAdamChunk, sg.n);
        if (skip) {  // a 16-bit gradient overflowed: drop the step, clear the gradients
            for (int64_t i = base + threadIdx.x; i < end; i += blockDim.x)
                sg.grad[i] = 0.f;
            continue;
        }
        const int64_t n_hash = sg.absmax ? sg.n_hash : 0;  // a multiple of 4: quadruples never straddle it
        // one quadruple of each array per thread (a 1024-float chunk is one pass of 256 threads)
        for (int64_t i = base + threadIdx.x * 4; i < end; i += blockDim.x * 4) {
            if (i + 4 <= end) {
                float4 th = *reinterpret_cast<float4 *>(sg.theta + i);
                const float4 g = __ldcs(reinterpret_cast<const float4 *>(sg.grad + i));
                float4 m = __ldcs(reinterpret_cast<const float4 *>(sg.m + i));
                float4 v = __ldcs(reinterpret_cast<const float4 *>(sg.v + i));
                adam_one(th.x, m.x, v.x, g.x, a.beta1, a.beta2, a.eps, lr_c1, inv_c2);
                adam_one(th.y, m.y, v.y, g.y, a.beta1, a.beta2, a.eps, lr_c1, inv_c2);
                adam_one(th.z, m.z, v.z, g.z, a.beta1, a.beta2, a.eps, lr_c1, inv_c2);
                adam_one(th.w, m.w, v.w, g.w, a.beta1, a.beta2, a.eps, lr_c1, inv_c2);
                *reinterpret_cast<float4 *>(sg.theta + i) = th;
                __stcs(reinterpret_cast<float4 *>(sg.m + i), m);
                __stcs(reinterpret_cast<float4 *>(sg.v + i), v);
                *reinterpret_cast<float4 *>(sg.grad + i) = make_float4(0.f, 0.f, 0.f, 0.f);
                if (i < n_hash)
                    amax = fmaxf(amax, fmaxf(fmaxf(fabsf(th.x), fabsf(th.y)), fmaxf(fabsf(th.z), fabsf(th.w))));
                if (sg.mirror && i < sg.n_hash)  // two entries of the tables' BF16 copy
                    *reinterpret_cast<uint2 *>(sg.mirror + i) = make_uint2(bf16_pair(th.x, th.y), bf16_pair(th.z, th.w));
            } else {
                for (int64_t j = i; j < end; ++j) {
                    adam_one(sg.theta[j], sg.m[j], sg.v[j], sg.grad[j], a.beta1, a.beta2, a.eps, lr_c1, inv_c2);
                    sg.grad[j] = 0.f;
                    if (j < n_hash)
                        amax = fmaxf(amax, fabsf(sg.theta[j]));
                    if (sg.mirror && j < sg.n_hash)
                        sg.mirror[j] = __bfloat16_as_ushort(__float2bfloat16_rn(sg.theta[j]));
                }
            }
        }
    }
    if (cur >= 0 && a.seg[cur].absmax)
        warp_absmax_to(a.seg[cur].absmax, amax);
}

cudaError_t launch_adam(const AdamArgs &a, int grid, cudaStream_t st)
{
    adam_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------- initialisation
// theta[i] = (2 u_i - 1) * bound, u_i from word 0 of Philox(ctr = (i lo, i hi,
// 'INIT', obj), key = seed); bound = 1e-4 for hash entries, sqrt(6 / (in + out))
// for MLP matrices (Xavier-uniform).
struct InitArgs {
    float *theta;
    int64_t n_hash;
    int32_t n_layers;
    int64_t layer_end[8];
    float bound[8];
    uint64_t seed;
    uint32_t obj;
};

__global__ void init_kernel(const InitArgs a)
{
    const int64_t n = a.layer_end[a.n_layers - 1];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float bound = 1e-4f;
        if (i >= a.n_hash) {
            int l = 0;
            while (l < a.n_layers - 1 && i >= a.layer_end[l])
                ++l;
            bound = a.bound[l];
        }
        const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0x494E4954u, a.obj),
                                      make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32)));
        a.theta[i] = (2.f * u24(r.x) - 1.f) * bound;
    }
}

cudaError_t launch_init_params(float *theta, int64_t n_hash, const int32_t *mlp_shape, int n_layers, uint64_t seed,
                               uint32_t obj, int grid, cudaStream_t st)
{
    if (n_layers < 1 || n_layers > 8)
        return cudaErrorInvalidValue;
    InitArgs a{};
    a.theta = theta;
    a.n_hash = n_hash;
    a.n_layers = n_layers;
    int64_t off = n_hash;
    for (int l = 0; l < n_layers; ++l) {
        const int out = mlp_shape[2 * l], in = mlp_shape[2 * l + 1];
        off += (int64_t)out * in;
        a.layer_end[l] = off;
        a.bound[l] = sqrtf(6.f / (float)(in + out));
    }
    a.seed = seed;
    a.obj = obj;
    init_kernel<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------ loss scaling
// Dynamic loss scale of a mixed-precision object, run after its Adam step:
// an overflow halves the scale (the step was dropped), growth_interval clean
// steps in a row double it (capped at 2^24).  An FP16 object's encoding scale
// then follows the tables and weights that Adam left (unchanged when the step
// was dropped, since theta was).
__device__ __forceinline__ float enc_scale_for(uint32_t absmax_bits, float gain)
{
    const float a = __uint_as_float(absmax_bits) * gain;
    if (!(a > 0.f))
        return ldexpf(1.f, kEncMaxLog2);  // an all-zero table: every scale is exact
    if (!isfinite(a))
        return 1.f;
    const int k = ilogbf(kEncTarget / a);  // floor(log2(kEncTarget / a)); INT_MAX for an infinite ratio
    return ldexpf(1.f, min(max(k, kEncMinLog2), kEncMaxLog2));
}

// max(1, max_l prod_{j<=l} ||W_j||_inf) over the hidden layers (all threads of
// the block call it and receive the value; one row per thread, width <= 128)
__device__ float mlp_gain(const LossScaleState *s)
{
    __shared__ uint32_t red[32];
    const float *w = s->mlp;
    int in = s->in;
    float cum = 1.f, gain = 1.f;
    for (int l = 0; l < s->hidden; ++l) {
        float rowsum = 0.f;
        if ((int)threadIdx.x < s->width)
            for (int c = 0; c < in; ++c)
                rowsum += fabsf(w[threadIdx.x * in + c]);
        const uint32_t m = __reduce_max_sync(kFull, __float_as_uint(rowsum));
        if ((threadIdx.x & 31) == 0)
            red[threadIdx.x >> 5] = m;
        __syncthreads();
        uint32_t bm = 0u;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i)
            bm = max(bm, red[i]);
        __syncthreads();
        cum *= __uint_as_float(bm);
        gain = fmaxf(gain, cum);
        w += (size_t)s->width * in;
        in = s->width;
    }
    return gain;
}

// The encoding scale from the gathered hash maximum and the weights (kept
// when `keep`); the gathered maximum restarts for the next pass.
__device__ void enc_update_block(LossScaleState *s, bool keep)
{
    if (!s->enc_auto)
        return;
    const float gain = mlp_gain(s);
    if (threadIdx.x == 0) {
        if (!keep)
            s->enc_scale = enc_scale_for(s->hash_absmax, gain);
        s->hash_absmax = 0u;
    }
}

// the scalar bookkeeping; returns whether the step was dropped
__device__ __forceinline__ bool loss_scale_update(LossScaleState *s)
{
    const bool dropped = s->overflow != 0;
    if (dropped) {
        s->scale = fmaxf(s->scale * 0.5f, 1.f);
        s->good_steps = 0;
        s->skipped += 1;
        s->overflow = 0;
    } else if (++s->good_steps >= s->growth_interval) {
        s->scale = fminf(s->scale * 2.f, 16777216.f);
        s->good_steps = 0;
    }
    return dropped;
}

constexpr int kScaleThreads = 128;  // one block per object: one MLP row per thread

// the bookkeeping of every object of l, one block each (the single-object path passes a list of one)
__global__ void __launch_bounds__(kScaleThreads) loss_scale_update_list_kernel(const ScaleList l)
{
    __shared__ int dropped;
    LossScaleState *s = l.s[blockIdx.x];
    if (threadIdx.x == 0)
        dropped = loss_scale_update(s);
    __syncthreads();
    enc_update_block(s, dropped != 0);
}

cudaError_t launch_loss_scale_update_list(const ScaleList &l, cudaStream_t st)
{
    if (l.n <= 0)
        return cudaSuccess;
    loss_scale_update_list_kernel<<<l.n, kScaleThreads, 0, st>>>(l);
    return cudaGetLastError();
}

cudaError_t launch_loss_scale_update(LossScaleState *s, cudaStream_t st)
{
    ScaleList l{};
    l.n = 1;
    l.s[0] = s;
    return launch_loss_scale_update_list(l, st);
}

// mirror[i] = bf16(theta[i]), i < n (n a multiple of 4; mirror 8-byte aligned)
__global__ void __launch_bounds__(256) mirror_kernel(const float *theta, int64_t n, uint16_t *mirror)
{
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; i < n; i += (int64_t)gridDim.x * blockDim.x * 4) {
        const float4 t = *reinterpret_cast<const float4 *>(theta + i);
        *reinterpret_cast<uint2 *>(mirror + i) = make_uint2(bf16_pair(t.x, t.y), bf16_pair(t.z, t.w));
    }
}

cudaError_t launch_mirror_refresh(const float *theta, int64_t n, uint16_t *mirror, int grid, cudaStream_t st)
{
    mirror_kernel<<<grid, 256, 0, st>>>(theta, n, mirror);
    return cudaGetLastError();
}

// max |theta[0..n_hash)| into s->hash_absmax; enc_scale_set_kernel then derives enc_scale from it
__global__ void __launch_bounds__(256) enc_absmax_kernel(const float *theta, int64_t n_hash, LossScaleState *s)
{
    float amax = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_hash; i += (int64_t)gridDim.x * blockDim.x)
        amax = fmaxf(amax, fabsf(theta[i]));
    warp_absmax_to(&s->hash_absmax, amax);
}

__global__ void __launch_bounds__(kScaleThreads) enc_scale_set_kernel(LossScaleState *s)
{
    enc_update_block(s, false);
}

cudaError_t launch_enc_scale_refresh(const float *theta, int64_t n_hash, LossScaleState *s, int grid,
                                     cudaStream_t st)
{
    enc_absmax_kernel<<<grid, 256, 0, st>>>(theta, n_hash, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    enc_scale_set_kernel<<<1, kScaleThreads, 0, st>>>(s);
    return cudaGetLastError();
}

__global__ void zero_losses_kernel(const WorkItem *items, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        *items[i].bd.loss = 0.f;
}

cudaError_t launch_zero_losses(const WorkItem *items, int n, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    zero_losses_kernel<<<(n + 127) / 128, 128, 0, st>>>(items, n);
    return cudaGetLastError();
}

size_t fused_tc_smem(int W, int IN, int H, bool split)
{
    switch (W * 100 + IN) {
    case 1608: return TcLayout<16, 8>::bytes(H, split);
    case 1616: return TcLayout<16, 16>::bytes(H, split);
    case 1632: return TcLayout<16, 32>::bytes(H, split);
    case 3208: return TcLayout<32, 8>::bytes(H, split);
    case 3216: return TcLayout<32, 16>::bytes(H, split);
    case 3232: return TcLayout<32, 32>::bytes(H, split);
    case 6408: return TcLayout<64, 8>::bytes(H, split);
    case 6416: return TcLayout<64, 16>::bytes(H, split);
    case 6432: return TcLayout<64, 32>::bytes(H, split);
    default: return 0;
    }
}

int fused_tc_occupancy_fp16(int W, int IN, int H, bool split);
int fused_tc_occupancy_bf16(int W, int IN, int H, bool split);

int fused_tc_occupancy(int precision, int W, int IN, int H, bool split)
{
    return precision == 2 ? fused_tc_occupancy_bf16(W, IN, H, split) : fused_tc_occupancy_fp16(W, IN, H, split);
}

static cudaError_t tc_dispatch(const WorkItem &one, const WorkList &wl, int W, int IN, int precision, int grid,
                               cudaStream_t st)
{
    if (precision == 1)
        return launch_fused_tc_fp16(one, wl, W, IN, grid, st);
    if (precision == 2)
        return launch_fused_tc_bf16(one, wl, W, IN, grid, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_fused_tc(const ObjDesc &od, const BatchDesc &bd, int precision, int grid, cudaStream_t st)
{
    WorkItem one{};
    one.od = od;
    one.bd = bd;
    one.tile_begin = 0;
    return tc_dispatch(one, WorkList{nullptr, 1, bd.n_tiles, od.H, bd.sp_x != nullptr}, od.W, od.IN, precision, grid,
                       st);
}

cudaError_t launch_fused_tc_list(const WorkList &wl, int W, int IN, int precision, int grid, cudaStream_t st)
{
    WorkItem unused{};
    return tc_dispatch(unused, wl, W, IN, precision, grid, st);
}

// ------------------------------------------------------- fused dispatch
size_t fused_fp32_smem(int W, int IN, int H, int S)
{
    return fused_fp32_smem_floats(W, IN, H, S) * sizeof(float);
}

int fused_fp32_pick_tile(int W, int IN, int H, size_t smem_limit)
{
    if (fused_fp32_smem(W, IN, H, 128) <= smem_limit)
        return 128;
    if (W == 64 && fused_fp32_smem(W, IN, H, 64) <= smem_limit)
        return 64;
    return 0;
}

static cudaError_t fp32_dispatch(const WorkItem &one, const WorkList &wl, int W, int IN, int S, int grid,
                                 cudaStream_t st)
{
    switch (W) {
    case 16: return launch_fused_fp32_w16(one, wl, IN, S, grid, st);
    case 32: return launch_fused_fp32_w32(one, wl, IN, S, grid, st);
    case 64: return launch_fused_fp32_w64(one, wl, IN, S, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_fused_fp32(const ObjDesc &od, const BatchDesc &bd, int S, int grid, cudaStream_t st)
{
    WorkItem one{};
    one.od = od;
    one.bd = bd;
    one.tile_begin = 0;
    return fp32_dispatch(one, WorkList{nullptr, 1, bd.n_tiles, od.H, bd.sp_x != nullptr}, od.W, od.IN, S, grid, st);
}

cudaError_t launch_fused_fp32_list(const WorkList &wl, int W, int IN, int S, int grid, cudaStream_t st)
{
    WorkItem unused{};
    return fp32_dispatch(unused, wl, W, IN, S, grid, st);
}

}  // namespace prenom
