// Training rays from RGB-D keyframes (§III-B "Training Data"): every pixel's
// camera ray in the object's normalised frame (box = unit cube), the pixels
// whose rays meet the box (and, on the object, have a depth) compacted in
// pixel order, and rays drawn uniformly from them.  The geometry is FP32 with
// every operation rounded explicitly (no contraction), so the candidate
// decisions and the outputs follow one fixed operation order.
#include "fused_fp32.cuh"
#include "prenom.h"

namespace prenom {

constexpr int kRayGenThreads = 256;
constexpr int kRayGenPerThread = 8;
constexpr int kRayGenChunk = kRayGenThreads * kRayGenPerThread;  // pixels per block of the scan

struct RayGenArgs {
    const prenom_keyframe *kf;  // device [n_kf]
    const int64_t *pix_off;     // device [n_kf + 1] first global pixel of each keyframe
    int32_t n_kf;
    int64_t n_pix;
    prenom_object_state st;
    int32_t *block_count;       // [n_blocks]
    int64_t *block_off;         // [n_blocks + 1]
    int32_t *cand;              // [n_pix] candidate pixels, in pixel order
    int64_t *n_cand;            // device scalar
    int32_t n_rays;
    const uint32_t *draws;      // [n_rays] or NULL: Philox words
    uint64_t seed;
    uint32_t call;
    float *o, *d, *rgb, *depth;
    uint8_t *is_obj;
};

__device__ __forceinline__ int kf_of_pixel(const RayGenArgs &a, int64_t p)
{
    int lo = 0, hi = a.n_kf - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.pix_off[mid] <= p)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// The object-frame ray of pixel (x, y); true when it is a candidate.
__device__ __forceinline__ bool pixel_ray(const prenom_keyframe &kf, const prenom_object_state &st, int x, int y,
                                          float (&o)[3], float (&d)[3], float (&rgb)[3], float &depth, uint8_t &obj)
{
    const float u = __fadd_rn((float)x, 0.5f), v = __fadd_rn((float)y, 0.5f);
    const float dc[3] = {__fdiv_rn(__fsub_rn(u, kf.cx), kf.fx), __fdiv_rn(__fsub_rn(v, kf.cy), kf.fy), 1.f};
    float dw[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        dw[a] = __fadd_rn(__fadd_rn(__fmul_rn(kf.R_wc[3 * a], dc[0]), __fmul_rn(kf.R_wc[3 * a + 1], dc[1])),
                          kf.R_wc[3 * a + 2]);
    const float nrm =
        __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(dw[0], dw[0]), __fmul_rn(dw[1], dw[1])), __fmul_rn(dw[2], dw[2])));
    float dh[3], rel[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dh[a] = __fdiv_rn(dw[a], nrm);
        rel[a] = __fsub_rn(kf.t_wc[a], st.centre[a]);
    }
    const float *Q = st.R_wo;  // object-to-world; its transpose maps world to object
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float ro = __fadd_rn(__fadd_rn(__fmul_rn(Q[a], rel[0]), __fmul_rn(Q[3 + a], rel[1])),
                                   __fmul_rn(Q[6 + a], rel[2]));
        const float rd = __fadd_rn(__fadd_rn(__fmul_rn(Q[a], dh[0]), __fmul_rn(Q[3 + a], dh[1])),
                                   __fmul_rn(Q[6 + a], dh[2]));
        o[a] = __fadd_rn(__fdiv_rn(ro, st.size[a]), 0.5f);
        d[a] = __fdiv_rn(rd, st.size[a]);
    }
    const int64_t pix = (int64_t)y * kf.width + x;
    obj = kf.mask[pix] == st.instance ? 1 : 0;
    const float D = kf.depth[pix];
    const bool valid = D > 0.f && isfinite(D);
#pragma unroll
    for (int c = 0; c < 3; ++c)
        rgb[c] = __fdiv_rn((float)kf.rgb[3 * pix + c], 255.f);
    depth = obj ? __fmul_rn(D, nrm) : 0.f;
    float tn, tf;
    return ray_box(o, d, tn, tf) && (!obj || valid);
}

__device__ __forceinline__ bool is_candidate(const RayGenArgs &a, int64_t p)
{
    if (p >= a.n_pix)
        return false;
    const int k = kf_of_pixel(a, p);
    const prenom_keyframe &kf = a.kf[k];
    const int64_t local = p - a.pix_off[k];
    float o[3], d[3], rgb[3], depth;
    uint8_t obj;
    return pixel_ray(kf, a.st, (int)(local % kf.width), (int)(local / kf.width), o, d, rgb, depth, obj);
}

__global__ void __launch_bounds__(kRayGenThreads) raygen_count_kernel(const RayGenArgs a)
{
    __shared__ int32_t s_cnt[kRayGenThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kRayGenChunk;
    int cnt = 0;
    for (int i = 0; i < kRayGenPerThread; ++i)
        cnt += is_candidate(a, base + (int64_t)i * kRayGenThreads + threadIdx.x) ? 1 : 0;
    cnt = __reduce_add_sync(kFull, (unsigned)cnt);
    if ((threadIdx.x & 31) == 0)
        s_cnt[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kRayGenThreads / 32; ++w)
            t += s_cnt[w];
        a.block_count[blockIdx.x] = t;
    }
}

// Exclusive offsets of the blocks' candidates and the total (one block).
__global__ void __launch_bounds__(1024) raygen_scan_kernel(const RayGenArgs a, int n_blocks)
{
    __shared__ int64_t s_part[1024];
    const int per = (n_blocks + 1023) / 1024;
    const int b0 = threadIdx.x * per, b1 = min(n_blocks, b0 + per);
    int64_t sum = 0;
    for (int b = b0; b < b1; ++b)
        sum += a.block_count[b];
    s_part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {  // 1024 partial sums in order
        int64_t run = 0;
        for (int t = 0; t < 1024; ++t) {
            const int64_t v = s_part[t];
            s_part[t] = run;
            run += v;
        }
        *a.n_cand = run;
        a.block_off[n_blocks] = run;
    }
    __syncthreads();
    int64_t run = s_part[threadIdx.x];
    for (int b = b0; b < b1; ++b) {
        a.block_off[b] = run;
        run += a.block_count[b];
    }
}

// Candidate pixels in pixel order: pass i of a block covers its pixels
// base + i*256 .. base + i*256 + 255, ranked by warp ballots and warp offsets.
__global__ void __launch_bounds__(kRayGenThreads) raygen_compact_kernel(const RayGenArgs a)
{
    __shared__ int32_t s_warp[kRayGenThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kRayGenChunk;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t out = a.block_off[blockIdx.x];
    for (int i = 0; i < kRayGenPerThread; ++i) {
        const int64_t p = base + (int64_t)i * kRayGenThreads + threadIdx.x;
        const bool c = is_candidate(a, p);
        const unsigned m = __ballot_sync(kFull, c);
        if (lane == 0)
            s_warp[warp] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < kRayGenThreads / 32; ++w) {
            before += w < warp ? s_warp[w] : 0;
            total += s_warp[w];
        }
        if (c)
            a.cand[out + before + __popc(m & ((1u << lane) - 1u))] = (int32_t)p;
        out += total;
        __syncthreads();
    }
}

// 32-bit word j of the internal stream: word j mod 4 of
// Philox4x32-10(ctr = (j / 4, 0, call, 0x52415953), key = seed).
__device__ __forceinline__ uint32_t raygen_word(uint64_t seed, uint32_t call, uint32_t j)
{
    const uint4 r = philox4x32_10(make_uint4(j >> 2, 0u, call, 0x52415953u),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    return pick(r, (int)(j & 3u));
}

__global__ void raygen_gather_kernel(const RayGenArgs a)
{
    const int64_t n = *a.n_cand;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < a.n_rays; j += gridDim.x * blockDim.x) {
        float o[3] = {-1.f, -1.f, -1.f}, d[3] = {0.f, 0.f, 0.f}, rgb[3] = {0.f, 0.f, 0.f}, depth = 0.f;
        uint8_t obj = 0;
        if (n > 0) {  // no candidate: a ray that misses the box and renders to zero
            const uint32_t r = a.draws ? a.draws[j] : raygen_word(a.seed, a.call, (uint32_t)j);
            const int64_t p = a.cand[(int64_t)(((uint64_t)r * (uint64_t)n) >> 32)];
            const int k = kf_of_pixel(a, p);
            const prenom_keyframe &kf = a.kf[k];
            const int64_t local = p - a.pix_off[k];
            pixel_ray(kf, a.st, (int)(local % kf.width), (int)(local / kf.width), o, d, rgb, depth, obj);
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a.o[3 * (int64_t)j + c] = o[c];
            a.d[3 * (int64_t)j + c] = d[c];
            a.rgb[3 * (int64_t)j + c] = rgb[c];
        }
        a.depth[j] = depth;
        a.is_obj[j] = obj;
    }
}

cudaError_t launch_make_rays(const prenom_keyframe *d_kf, const int64_t *d_pix_off, int n_kf, int64_t n_pix,
                             const prenom_object_state &st, unsigned char *scratch, int n_rays, const uint32_t *draws,
                             uint64_t seed, uint32_t call, float *o, float *d, float *rgb, float *depth,
                             uint8_t *is_obj, int64_t **d_count, cudaStream_t st_)
{
    RayGenArgs a{};
    a.kf = d_kf;
    a.pix_off = d_pix_off;
    a.n_kf = n_kf;
    a.n_pix = n_pix;
    a.st = st;
    const int n_blocks = (int)((n_pix + kRayGenChunk - 1) / kRayGenChunk);
    unsigned char *p = scratch;
    a.n_cand = reinterpret_cast<int64_t *>(p);
    p += 256;
    a.block_off = reinterpret_cast<int64_t *>(p);
    p += ((size_t)(n_blocks + 1) * sizeof(int64_t) + 255) / 256 * 256;
    a.block_count = reinterpret_cast<int32_t *>(p);
    p += ((size_t)n_blocks * sizeof(int32_t) + 255) / 256 * 256;
    a.cand = reinterpret_cast<int32_t *>(p);
    a.n_rays = n_rays;
    a.draws = draws;
    a.seed = seed;
    a.call = call;
    a.o = o;
    a.d = d;
    a.rgb = rgb;
    a.depth = depth;
    a.is_obj = is_obj;
    *d_count = a.n_cand;
    if (n_blocks > 0) {
        raygen_count_kernel<<<n_blocks, kRayGenThreads, 0, st_>>>(a);
        raygen_scan_kernel<<<1, 1024, 0, st_>>>(a, n_blocks);
        raygen_compact_kernel<<<n_blocks, kRayGenThreads, 0, st_>>>(a);
    } else {
        cudaMemsetAsync(a.n_cand, 0, sizeof(int64_t), st_);
    }
    if (n_rays > 0)
        raygen_gather_kernel<<<(n_rays + 255) / 256, 256, 0, st_>>>(a);
    return cudaGetLastError();
}

size_t make_rays_scratch(int64_t n_pix)
{
    const int64_t n_blocks = (n_pix + kRayGenChunk - 1) / kRayGenChunk;
    return 256 + ((size_t)(n_blocks + 1) * sizeof(int64_t) + 255) / 256 * 256 +
           ((size_t)n_blocks * sizeof(int32_t) + 255) / 256 * 256 + (size_t)n_pix * sizeof(int32_t);
}

}  // namespace prenom
