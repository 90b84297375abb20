// Device helpers of the fused PRENOM kernels: counter-based random numbers,
// error-free position arithmetic, hash-grid indexing, prior-grid lookup and warp scans.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "prenom_internal.h"

namespace prenom {

constexpr unsigned kFull = 0xffffffffu;

// Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC 2011).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ float u24(uint32_t x) { return (float)(x >> 8) * 5.9604644775390625e-8f; }

__device__ __forceinline__ uint32_t pick(uint4 v, int i)
{
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// Stratified uniform u_{r,k} = (k + xi) / nr in IEEE single precision, xi the
// top 17 bits of word k mod 4 of Philox(ctr = (ray, k div 4, step, 2 obj),
// key = seed) times 2^-17: k + xi is then exact for k < 128, so u < 1.
__device__ __forceinline__ float philox_uniform(uint64_t seed, uint32_t step, uint32_t obj, uint32_t ray,
                                                int k, int nr)
{
    const uint4 o = philox4x32_10(make_uint4(ray, (uint32_t)k >> 2, step, 2u * obj),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const float xi = (float)(pick(o, k & 3) >> 15) * 7.62939453125e-06f;
    return __fdiv_rn(__fadd_rn((float)k, xi), (float)nr);
}

// Background colour C_rand of a ray: words 0..2 of Philox(ctr = (ray, 0, step, 2 obj + 1)).
__device__ __forceinline__ float3 philox_colour(uint64_t seed, uint32_t step, uint32_t obj, uint32_t ray)
{
    const uint4 o = philox4x32_10(make_uint4(ray, 0u, step, 2u * obj + 1u),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    return make_float3(u24(o.x), u24(o.y), u24(o.z));
}

// p = o + t d as an unevaluated sum hi + lo (error-free product and sum), so
// that the cell coordinates p N_l keep ~48 bits even at N_l = 2048.
__device__ __forceinline__ void pos_two_float(float o, float t, float d, float &hi, float &lo)
{
    const float p = __fmul_rn(t, d);
    const float pe = __fmaf_rn(t, d, -p);  // exact error of the product
    const float s = __fadd_rn(o, p);
    const float bb = __fsub_rn(s, o);
    const float se = __fadd_rn(__fsub_rn(o, __fsub_rn(s, bb)), __fsub_rn(p, bb));  // exact error of the sum
    const float l = __fadd_rn(se, pe);
    hi = __fadd_rn(s, l);
    lo = __fsub_rn(l, __fsub_rn(hi, s));
    // clamp to the unit cube (a NaN position maps to the origin)
    if (!(hi >= 0.f) || (hi == 0.f && lo < 0.f)) {
        hi = 0.f;
        lo = 0.f;
    } else if (hi > 1.f || (hi == 1.f && lo > 0.f)) {
        hi = 1.f;
        lo = 0.f;
    }
}

// Cell c0 = min(floor(p N), N - 1) and local coordinate w = p N - c0 in [0, 1]
// from p = hi + lo.
__device__ __forceinline__ void level_cell(float hi, float lo, int N, int &c0, float &w)
{
    const float nf = (float)N;
    const float s = __fmul_rn(hi, nf);
    const float se = __fmaf_rn(hi, nf, -s);  // exact error of hi * N
    const float sl = __fmaf_rn(lo, nf, se);
    float f = floorf(s);
    float fr = __fadd_rn(__fsub_rn(s, f), sl);  // s - f is exact
    if (fr < 0.f) {
        f -= 1.f;
        fr = __fadd_rn(fr, 1.f);
    } else if (fr >= 1.f) {
        f += 1.f;
        fr = __fsub_rn(fr, 1.f);
    }
    if (f < 0.f) {
        f = 0.f;
        fr = 0.f;
    }
    if (f > nf - 1.f) {
        fr = __fadd_rn(fr, f - (nf - 1.f));
        f = nf - 1.f;
    }
    c0 = (int)f;
    w = fr;
}

constexpr uint32_t kPi2 = 2654435761u;
constexpr uint32_t kPi3 = 805459861u;

// Entry of vertex (x, y, z) on a level: dense (x fastest) or spatial hash mod T.
__device__ __forceinline__ uint32_t grid_index(bool dense, uint32_t n1, uint32_t tmask, uint32_t x, uint32_t y,
                                               uint32_t z)
{
    return dense ? x + n1 * (y + n1 * z) : ((x ^ (y * kPi2) ^ (z * kPi3)) & tmask);
}

// The 8 corner entries and trilinear weights of point (hi+lo) on level lv.
struct Corners {
    uint32_t idx[8];
    float wt[8];
    int cell[3];  // lower corner of the cell
};

__device__ __forceinline__ void level_corners(const LevelDesc &lv, uint32_t tmask, const float (&ph)[3],
                                              const float (&pl)[3], Corners &cs)
{
    int c[3];
    float w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
        level_cell(ph[a], pl[a], lv.res, c[a], w[a]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
        cs.cell[a] = c[a];
    const uint32_t n1 = (uint32_t)lv.res + 1u;
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
        const int bx = corner & 1, by = (corner >> 1) & 1, bz = (corner >> 2) & 1;
        const float wx = bx ? w[0] : 1.f - w[0];
        const float wy = by ? w[1] : 1.f - w[1];
        const float wz = bz ? w[2] : 1.f - w[2];
        cs.wt[corner] = __fmul_rn(__fmul_rn(wx, wy), wz);
    }
    // the level's storage is uniform across the warp: one branch, one index formula
    const uint32_t x = (uint32_t)c[0], y = (uint32_t)c[1], z = (uint32_t)c[2];
    if (lv.dense) {
#pragma unroll
        for (int corner = 0; corner < 8; ++corner)
            cs.idx[corner] = grid_index(true, n1, tmask, x + (corner & 1), y + ((corner >> 1) & 1),
                                        z + ((corner >> 2) & 1));
    } else {
#pragma unroll
        for (int corner = 0; corner < 8; ++corner)
            cs.idx[corner] = grid_index(false, n1, tmask, x + (corner & 1), y + ((corner >> 1) & 1),
                                        z + ((corner >> 2) & 1));
    }
}

// Bounds checks of a PRENOM_DEBUG_BOUNDS build.  The regular build has none: its
// indices are in range by construction (positions clamped to the unit cube,
// cells to [0, N_l - 1], hashes masked to T - 1, rays and tiles counted from the
// batch).  The debug build tests each table, grid and ray index where it is
// formed; an index outside its array sets kStatusBounds in the status word
// (prenom_sync then returns PRENOM_ERR_DEVICE_BOUNDS) and its access is
// skipped, never a trap or a fault.
#ifdef PRENOM_DEBUG_BOUNDS
__device__ __forceinline__ bool bounds_ok(bool ok, int32_t *status)
{
    if (!ok && status)
        atomicOr(status, kStatusBounds);
    return ok;
}

// Each corner must address an entry of its level: (N_l + 1)^3 entries when dense,
// T when hashed.  An entry outside is replaced by entry 0 with weight 0.
__device__ __forceinline__ void check_corners(const LevelDesc &lv, uint32_t tmask, Corners &cs, int32_t *status)
{
    const uint32_t n1 = (uint32_t)lv.res + 1u;
    const uint32_t n = lv.dense ? n1 * n1 * n1 : tmask + 1u;
#pragma unroll
    for (int c = 0; c < 8; ++c)
        if (!bounds_ok(cs.idx[c] < n, status)) {
            cs.idx[c] = 0u;
            cs.wt[c] = 0.f;
        }
}
#define PRENOM_CHECK_CORNERS(lv, tmask, cs, status) check_corners(lv, tmask, cs, status)
#define PRENOM_BOUNDS_OK(cond, status) bounds_ok((cond), (status))
#else
#define PRENOM_CHECK_CORNERS(lv, tmask, cs, status) ((void)0)
#define PRENOM_BOUNDS_OK(cond, status) true
#endif

// Prior density at x: trilinear over voxel centres, g = x R - 1/2 clamped to [0, R-1].
__device__ __forceinline__ float prior_lookup(const float *__restrict__ grid, int R, float x, float y, float z,
                                              int32_t *status = nullptr)
{
    const float rf = (float)R;
    const float q[3] = {x, y, z};
    int c[3];
    float w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float g = __fmaf_rn(q[a], rf, -0.5f);
        g = fminf(fmaxf(g, 0.f), rf - 1.f);
        float f = fminf(floorf(g), rf - 2.f);
        c[a] = (int)f;
        w[a] = g - f;
    }
    float s = 0.f;
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
        const int bx = corner & 1, by = (corner >> 1) & 1, bz = (corner >> 2) & 1;
        const float wt = (bx ? w[0] : 1.f - w[0]) * (by ? w[1] : 1.f - w[1]) * (bz ? w[2] : 1.f - w[2]);
        const size_t vox = ((size_t)(c[2] + bz) * R + (c[1] + by)) * R + (c[0] + bx);
        if (!PRENOM_BOUNDS_OK(vox < (size_t)R * R * R, status))
            continue;
        const float v = __ldg(grid + vox);
        s += (wt == 0.f) ? 0.f : wt * v;
    }
    return s;
}

// Raises a kernel's dynamic shared-memory limit to all the device allows beside
// its static shared memory.  The limit is a permission, not a reservation (each
// launch takes what it asks for), and a limit that only grows keeps every
// earlier launch of the kernel valid: a CUDA graph captured with a larger
// launch (an object with more hidden layers) stays launchable after a later,
// smaller launch of the same kernel, also where a tool relaunches graph nodes
// one by one.
template <typename K>
cudaError_t allow_max_dynamic_smem(K kern)
{
    cudaFuncAttributes fa{};
    int dev = 0, optin = 0;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e == cudaSuccess)
        e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
}

// Fire-and-forget reductions into global memory.  The explicit .global state
// space matters: a pointer read from a descriptor is otherwise a generic
// address, and generic atomics are ordered against shared-memory traffic.
__device__ __forceinline__ void red_add_f2(float2 *p, float a, float b)
{
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(__cvta_generic_to_global(p)), "f"(a), "f"(b));
}

__device__ __forceinline__ void red_add_f4(float4 *p, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(__cvta_generic_to_global(p)), "f"(a),
                 "f"(b), "f"(c), "f"(d));
}

// Corners 2j and 2j+1 differ only in x.  When their entries differ only in
// bit 0 they share one 16-byte-aligned pair of entries (every level starts on
// a multiple of 8 two-feature entries and the table base is 16-byte aligned),
// so one 16-byte access serves both.  At hashed levels this holds for every
// even x (the x prime is 1); at dense levels for every even flat index.
__device__ __forceinline__ void gather_pair(const float2 *tab, uint32_t i0, uint32_t i1, float2 &f0, float2 &f1)
{
    if ((i0 ^ i1) == 1u) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(tab + (i0 & ~1u)));
        const bool first = (i0 & 1u) == 0u;
        f0 = first ? make_float2(q.x, q.y) : make_float2(q.z, q.w);
        f1 = first ? make_float2(q.z, q.w) : make_float2(q.x, q.y);
    } else {
        f0 = __ldg(tab + i0);
        f1 = __ldg(tab + i1);
    }
}

// One entry of a BF16 table: a 32-bit word, feature 0 in the low half (a bf16
// is the top half of the FP32 it rounds, so widening is a shift).
__device__ __forceinline__ float2 bf16x2_entry(uint32_t w)
{
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
}

// Two entries of a BF16 table.  x-adjacent corners whose indices differ only in
// their two low bits lie in one aligned group of four entries (16 bytes; every
// level starts on a multiple of 8 entries), so one load serves both: at hashed
// levels for x = 0, 1, 2 mod 4 (the x prime is 1), at dense levels for flat
// indices 0, 1, 2 mod 4 -- three pairs in four, against one in two for the
// 8-byte FP32 entries.
__device__ __forceinline__ void gather_pair16(const uint32_t *tab, uint32_t i0, uint32_t i1, float2 &f0, float2 &f1)
{
    if ((i0 ^ i1) < 4u) {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(tab + (i0 & ~3u)));
        const uint32_t k0 = i0 & 3u, k1 = i1 & 3u;
        const uint32_t w0 = k0 == 0u ? q.x : k0 == 1u ? q.y : k0 == 2u ? q.z : q.w;
        const uint32_t w1 = k1 == 0u ? q.x : k1 == 1u ? q.y : k1 == 2u ? q.z : q.w;
        f0 = bf16x2_entry(w0);
        f1 = bf16x2_entry(w1);
    } else {
        f0 = bf16x2_entry(__ldg(tab + i0));
        f1 = bf16x2_entry(__ldg(tab + i1));
    }
}

// Adds (a0, a1) to entry i0 and (b0, b1) to entry i1, skipping an entry whose
// two addends are zero (an exact zero where the pair is one access).
__device__ __forceinline__ void scatter_pair(float2 *gtab, uint32_t i0, uint32_t i1, float a0, float a1, float b0,
                                             float b1)
{
    const bool ua = a0 != 0.f || a1 != 0.f, ub = b0 != 0.f || b1 != 0.f;
    if ((i0 ^ i1) == 1u) {
        if (ua || ub) {
            const bool first = (i0 & 1u) == 0u;
            red_add_f4(reinterpret_cast<float4 *>(gtab + (i0 & ~1u)), first ? a0 : b0, first ? a1 : b1,
                       first ? b0 : a0, first ? b1 : a1);
        }
    } else {
        if (ua)
            red_add_f2(gtab + i0, a0, a1);
        if (ub)
            red_add_f2(gtab + i1, b0, b1);
    }
}

// Hash-grid scatter of one level for the 32 samples of a warp (all lanes call
// it together; inactive lanes add nothing).  dL/d(entry) of corner c is the sum
// over samples of w_c(x) (g0, g1).  Samples of a ray sit in depth order in
// consecutive lanes, so at coarse levels runs of lanes share one cell: a
// segmented warp scan sums each run (in chunks, below) first and only the
// chunk's last lane issues the reductions.  A corner of zero weight adds nothing.
// Lanes of one cell are summed in chunks of at most 2^CHUNK_LOG2 lanes (5 is a
// whole run) before the reductions: fewer shuffle rounds against more
// reductions.  Measured on the full-size single object, the scatter kernel
// takes 96.5 / 74.8 / 75.5 / 78.9 / 82.6 us for chunks of 1 / 2 / 4 / 8 / 32
// lanes and the whole step is fastest with 4; on the 32-object batched step
// (smaller tables, more reductions per entry) 1642 / 1447 / 1355 / 1314 us for
// 2 / 4 / 8 / 32, so the split form's scatter comes in both, chosen by the
// autotuner.
constexpr int kScatterChunkLog2 = 2;

template <int CHUNK_LOG2 = kScatterChunkLog2>
__device__ __forceinline__ void scatter_level_warp(float2 *gtab, bool active, const Corners &cs, float g0, float g1,
                                                   int lane)
{
    const int k0 = active ? cs.cell[0] : -1 - lane;  // inactive lanes match no neighbour
    const int k1 = active ? cs.cell[1] : 0, k2 = active ? cs.cell[2] : 0;
    const int p0 = __shfl_up_sync(kFull, k0, 1), p1 = __shfl_up_sync(kFull, k1, 1), p2 = __shfl_up_sync(kFull, k2, 1);
    const bool head = lane == 0 || p0 != k0 || p1 != k1 || p2 != k2;
    uint32_t heads = __ballot_sync(kFull, head);
    const uint32_t upto = 0xffffffffu >> (31 - lane);  // lanes 0..lane
    int pos = lane - (31 - __clz(heads & upto));  // position in the run
    if constexpr (CHUNK_LOG2 < 5) {  // runs cut into chunks of 2^CHUNK_LOG2 lanes
        heads |= __ballot_sync(kFull, (pos & ((1 << CHUNK_LOG2) - 1)) == 0);
        pos = lane - (31 - __clz(heads & upto));
    }
    const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u) != 0u;
    float v[16];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const bool use = active && cs.wt[c] != 0.f;
        v[2 * c] = use ? cs.wt[c] * g0 : 0.f;
        v[2 * c + 1] = use ? cs.wt[c] * g1 : 0.f;
    }
    if (heads != 0xffffffffu) {
        const int maxpos = (int)__reduce_max_sync(kFull, (unsigned)pos);
        for (int d = 1; d <= maxpos; d <<= 1) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const float up = __shfl_up_sync(kFull, v[q], d);
                if (pos >= d)
                    v[q] += up;
            }
        }
    }
    if (active && tail) {
#pragma unroll
        for (int c = 0; c < 8; c += 2)
            scatter_pair(gtab, cs.idx[c], cs.idx[c + 1], v[2 * c], v[2 * c + 1], v[2 * c + 2], v[2 * c + 3]);
    }
}

__device__ __forceinline__ void red_add_f(float *p, float a)
{
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "f"(a));
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1)
        v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ float warp_incl_scan(float v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float n = __shfl_up_sync(kFull, v, o);
        if (lane >= o)
            v += n;
    }
    return v;
}

// Inclusive suffix scan: lane i gets the sum of lanes i..31.
__device__ __forceinline__ float warp_incl_suffix(float v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float n = __shfl_down_sync(kFull, v, o);
        if (lane + o < 32)
            v += n;
    }
    return v;
}

}  // namespace prenom
