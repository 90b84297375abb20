// Fused FP32 training step of one object NeRF on sm_103a.
//
// One persistent CTA (256 threads) per SM walks tiles of whole rays.  A tile
// holds S samples (S = 128 or 64) as rows of shared-memory activation
// matrices stored feature-major ([feature][sample], row stride S + 4 floats),
// so every stage of the step reads its operands from shared memory and no
// per-sample intermediate ever goes to HBM:
//   1. ray setup and prior sampling, one warp per ray (§III-B "Probabilistic
//      Ray Sampling": probes, Eq. 4-6 via a warp scan of sigma*delta, escape
//      rule, inverse transform by binary search over the CDF in shared memory);
//   2. hash-grid encoding, two (or four) threads per sample, levels split
//      between them, with error-free position arithmetic;
//   3. MLP forward as register-tiled FFMA GEMMs over the tile;
//   4. compositing (Eq. 7), loss (Eq. 8-9) and its adjoint, one warp per 32
//      samples of a ray, one sample per lane, with shuffle scans (prefix for
//      transmittance, suffix for the adjoint) joined across a ray's warps;
//   5. MLP backward: dW accumulated in shared memory across all tiles of the
//      CTA (flushed once with atomics at the end), dX by GEMM;
//   6. hash-grid scatter of dX: runs of lanes in one cell summed by a
//      segmented warp scan, then vector reductions (one 16-byte reduction for
//      an x-adjacent corner pair that shares an aligned entry pair).
#pragma once

#include "device_common.cuh"

namespace prenom {

// Per-ray fields kept in shared memory during a tile.
enum RayField { RF_O = 0, RF_D = 3, RF_RGB = 6, RF_DEPTH = 9, RF_OBJ = 10, RF_CR = 11, RF_TN = 14, RF_TF = 15 };
constexpr int kRayStride = 16;

enum Epi { kStore = 0, kRelu = 1, kMaskByOld = 2 };

template <int R>
__device__ __forceinline__ void ld_vec(const float *p, float (&v)[R])
{
    if constexpr (R == 8) {
        const float4 a = *reinterpret_cast<const float4 *>(p), b = *reinterpret_cast<const float4 *>(p + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else if constexpr (R == 4) {
        const float4 a = *reinterpret_cast<const float4 *>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    } else if constexpr (R == 2) {
        const float2 a = *reinterpret_cast<const float2 *>(p);
        v[0] = a.x; v[1] = a.y;
    } else {
#pragma unroll
        for (int i = 0; i < R; ++i)
            v[i] = p[i];
    }
}

template <int R>
__device__ __forceinline__ void st_vec(float *p, const float (&v)[R])
{
    if constexpr (R == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    } else {
#pragma unroll
        for (int i = 0; i < R; ++i)
            p[i] = v[i];
    }
}

// C_T[n][s] = epi( sum_k A_T[k][s] * B[k][n] ) for the tile's S samples and N
// outputs.  A_T, C_T: [.][S+4]; B: [K][N].  Each thread owns S/32 samples x N/8
// outputs; a warp covers 8 sample groups x 4 output groups, so operand loads
// are single-wavefront broadcasts and stores fill whole 128-byte rows.
template <int S, int N, int EPI>
__device__ __forceinline__ void gemm_sn(const float *__restrict__ AT, const float *__restrict__ B, int K,
                                        float *CT)
{
    constexpr int SP = S + 4;
    constexpr int RM = S / 32;
    constexpr int RN = N / 8;
    static_assert(RN >= 1 && RM >= 1, "tile shape");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cg = (warp & 1) * 4 + (lane & 3);
    const int rg = (warp >> 1) * 8 + (lane >> 2);
    const int s0 = rg * RM, n0 = cg * RN;
    float acc[RM][RN];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j)
            acc[i][j] = 0.f;
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        float a[RM], b[RN];
        ld_vec<RM>(AT + k * SP + s0, a);
        ld_vec<RN>(B + k * N + n0, b);
#pragma unroll
        for (int i = 0; i < RM; ++i)
#pragma unroll
            for (int j = 0; j < RN; ++j)
                acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
#pragma unroll
    for (int j = 0; j < RN; ++j) {
        float *c = CT + (n0 + j) * SP + s0;
        float v[RM];
        if constexpr (EPI == kMaskByOld) {
            float old[RM];
            ld_vec<RM>(c, old);
#pragma unroll
            for (int i = 0; i < RM; ++i)
                v[i] = old[i] > 0.f ? acc[i][j] : 0.f;
        } else {
#pragma unroll
            for (int i = 0; i < RM; ++i)
                v[i] = (EPI == kRelu) ? fmaxf(acc[i][j], 0.f) : acc[i][j];
        }
        st_vec<RM>(c, v);
    }
}

template <int N, int K>
struct DwShape {
    static constexpr int total = N * K;
    static constexpr int per = total >= kThreads ? total / kThreads : 1;
    static constexpr int rn0 = per >= 16 ? 4 : (per >= 4 ? 2 : (per >= 2 && N >= K ? 2 : 1));
    static constexpr int RN = rn0 > N ? N : rn0;
    static constexpr int RK = per / RN > K ? K : (per / RN < 1 ? 1 : per / RN);
    static constexpr int TN = N / RN, TK = K / RK;
    static_assert(TN * TK <= kThreads, "dW tile");
    static_assert(RN * RK * TN * TK == total, "dW cover");
};

// D[n][k] += sum_s A_T[n][s] * B_T[k][s] (weight gradient of one layer over the
// tile's samples).  D is row-major [N][K] in shared memory and every entry has
// exactly one owning thread, so the update needs no atomics.  Rows owned by a
// thread are interleaved (n = ni + i*TN) so a phase of 8 lanes reads 8
// consecutive rows: with the +4 row padding these hit disjoint banks.
template <int S, int N, int K>
__device__ __forceinline__ void gemm_dw(const float *__restrict__ AT, const float *__restrict__ BT, float *D)
{
    using Sh = DwShape<N, K>;
    constexpr int SP = S + 4;
    const int tid = threadIdx.x;
    if (tid >= Sh::TN * Sh::TK)
        return;
    const int ki = tid % Sh::TK, ni = tid / Sh::TK;
    float acc[Sh::RN][Sh::RK];
#pragma unroll
    for (int i = 0; i < Sh::RN; ++i)
#pragma unroll
        for (int j = 0; j < Sh::RK; ++j)
            acc[i][j] = 0.f;
#pragma unroll 2
    for (int s = 0; s < S; s += 4) {
        float4 a[Sh::RN], b[Sh::RK];
#pragma unroll
        for (int i = 0; i < Sh::RN; ++i)
            a[i] = *reinterpret_cast<const float4 *>(AT + (ni + i * Sh::TN) * SP + s);
#pragma unroll
        for (int j = 0; j < Sh::RK; ++j)
            b[j] = *reinterpret_cast<const float4 *>(BT + (ki + j * Sh::TK) * SP + s);
#pragma unroll
        for (int i = 0; i < Sh::RN; ++i)
#pragma unroll
            for (int j = 0; j < Sh::RK; ++j) {
                float t = acc[i][j];
                t = fmaf(a[i].x, b[j].x, t);
                t = fmaf(a[i].y, b[j].y, t);
                t = fmaf(a[i].z, b[j].z, t);
                t = fmaf(a[i].w, b[j].w, t);
                acc[i][j] = t;
            }
    }
#pragma unroll
    for (int i = 0; i < Sh::RN; ++i)
#pragma unroll
        for (int j = 0; j < Sh::RK; ++j)
            D[(ni + i * Sh::TN) * K + ki + j * Sh::TK] += acc[i][j];
}

// Output layer forward: O_T[o][s] = sum_i H_T[i][s] * Wf_out[i][o], o < 4.
template <int W, int S>
__device__ __forceinline__ void out_layer_fwd(const float *__restrict__ HTl, const float *__restrict__ Wfo, float *OT)
{
    constexpr int SP = S + 4;
    constexpr int PARTS = kThreads / S;
    constexpr int OPT = 4 / PARTS;
    const int s = threadIdx.x % S, og = threadIdx.x / S;
    float acc[OPT];
#pragma unroll
    for (int j = 0; j < OPT; ++j)
        acc[j] = 0.f;
#pragma unroll 8
    for (int i = 0; i < W; ++i) {
        const float h = HTl[i * SP + s];
#pragma unroll
        for (int j = 0; j < OPT; ++j)
            acc[j] = fmaf(h, Wfo[i * 4 + og * OPT + j], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < OPT; ++j)
        OT[(og * OPT + j) * SP + s] = acc[j];
}

// ---------------------------------------------------------------- sampling
// One warp samples one ray: slab intersection with the unit cube, nc probes at
// bin centres, sigma = prior density (trilinear), s_i = sum_{j<=i} sigma_j delta
// by a warp scan, sum_{j<=i} rho_term_j = 1 - exp(-s_i) (the telescoped form of
// Eq. 5), CDF of Eq. 6, uniform CDF i/nc for escaping rays, then for each
// uniform the first bin b with CDF(b+1) > u and a linear position inside it.
// Slab intersection of the ray o + t d (t >= 0) with the unit cube: [tn, tf],
// or tn = tf = 0 for a ray that misses it.
__device__ __forceinline__ bool ray_box(const float (&o)[3], const float (&d)[3], float &tn, float &tf)
{
    float t0 = 0.f, t1 = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (d[a] != 0.f) {
            const float ta = __fdiv_rn(0.f - o[a], d[a]);
            const float tb = __fdiv_rn(1.f - o[a], d[a]);
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
        } else if (o[a] < 0.f || o[a] > 1.f) {
            t1 = -INFINITY;
        }
    }
    const bool hit = t1 > t0;
    tn = hit ? t0 : 0.f;
    tf = hit ? t1 : 0.f;
    return hit;
}

__device__ __forceinline__ void sample_ray_warp(const ObjDesc &od, const BatchDesc &bd, int r, int gr, float *rf,
                                                float *ts, float *cdf, int lane)
{
    const int nc = bd.nc, nr = bd.nr;
    const float o[3] = {rf[RF_O], rf[RF_O + 1], rf[RF_O + 2]};
    const float d[3] = {rf[RF_D], rf[RF_D + 1], rf[RF_D + 2]};
    float tn, tf;
    const bool hit = ray_box(o, d, tn, tf);
    if (lane == 0) {
        rf[RF_TN] = tn;
        rf[RF_TF] = tf;
    }
    const int Q = (nr + 31) >> 5;
    if (bd.t_in) {
        for (int q = 0; q < Q; ++q) {
            const int k = lane * Q + q;
            if (k < nr) {
                const float t = bd.t_in[(size_t)gr * nr + k];
                ts[r * nr + k] = t;
                if (bd.out_t)
                    bd.out_t[(size_t)gr * nr + k] = t;
                if (bd.out_bins)
                    bd.out_bins[(size_t)gr * nr + k] = -1;
            }
        }
        return;
    }
    const float delta = __fdiv_rn(tf - tn, (float)nc);
    const int Qc = (nc + 31) >> 5;
    float inc[kMaxNc / 32];
    float run = 0.f;
#pragma unroll
    for (int q = 0; q < kMaxNc / 32; ++q) {
        if (q < Qc) {
            const int i = lane * Qc + q;
            float tau = 0.f;
            if (hit && i < nc) {
                const float ti = __fmaf_rn((float)i + 0.5f, delta, tn);
                const float sig = prior_lookup(od.grid, od.R, __fmaf_rn(ti, d[0], o[0]), __fmaf_rn(ti, d[1], o[1]),
                                               __fmaf_rn(ti, d[2], o[2]), bd.status);
                tau = sig * delta;
            }
            run += tau;
            inc[q] = run;
        }
    }
    const float incl = warp_incl_scan(run, lane);
    float base = __shfl_up_sync(kFull, incl, 1);
    if (lane == 0)
        base = 0.f;
    const float s_total = __shfl_sync(kFull, incl, 31);
    const float total = -expm1f(-s_total);
    const bool escape = !(total >= bd.escape_eps);
#pragma unroll
    for (int q = 0; q < kMaxNc / 32; ++q) {
        if (q < Qc) {
            const int i = lane * Qc + q;
            if (i < nc - 1) {
                const float ci = -expm1f(-(base + inc[q]));
                cdf[i + 1] = escape ? __fdiv_rn((float)(i + 1), (float)nc) : __fdiv_rn(ci, total);
            }
        }
    }
    if (lane == 0) {
        cdf[0] = 0.f;
        cdf[nc] = 1.f;
    }
    __syncwarp();
    for (int q = 0; q < Q; ++q) {
        const int k = lane * Q + q;
        if (k < nr) {
            float u = bd.u ? bd.u[(size_t)gr * nr + k] : philox_uniform(bd.seed, bd.step, bd.obj_id, gr, k, nr);
            u = fminf(fmaxf(u, 0.f), 0x1.fffffep-1f);  // a caller's uniform outside [0, 1) is clamped
            int lo = 0, hi = nc - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (cdf[mid + 1] > u)
                    hi = mid;
                else
                    lo = mid + 1;
            }
            const float c0 = cdf[lo], c1 = cdf[lo + 1];
            const float frac = c1 > c0 ? fminf(__fdiv_rn(u - c0, c1 - c0), 1.f) : 0.f;
            const float t = __fmaf_rn((float)lo + frac, delta, tn);
            ts[r * nr + k] = t;
            if (bd.out_t)
                bd.out_t[(size_t)gr * nr + k] = t;
            if (bd.out_bins)
                bd.out_bins[(size_t)gr * nr + k] = lo;
        }
    }
    __syncwarp();
}

// ---------------------------------------------------------------- encoding
// Thread (s, part) encodes levels part, part + PARTS, ... of sample s.  Rows of
// samples beyond the tile's valid count are zeroed (they stay inert through
// the GEMMs and are never scattered).
template <int IN, int S, bool SCATTER>
__device__ __forceinline__ void encode_or_scatter(const ObjDesc &od, const BatchDesc &bd, const float *rayf,
                                                  const float *ts, float *XT, float *dOT, int ns)
{
    constexpr int SP = S + 4;
    constexpr int PARTS = kThreads / S;
    constexpr int L = IN / 2;
    static_assert(S % 32 == 0, "a warp holds consecutive samples of one part");
    const int s = threadIdx.x % S, part = threadIdx.x / S;
    const bool active = s < ns;
    if constexpr (!SCATTER) {
        if (!active) {
            for (int l = part; l < L; l += PARTS) {
                XT[(2 * l) * SP + s] = 0.f;
                XT[(2 * l + 1) * SP + s] = 0.f;
            }
            if (part == 0) {
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    dOT[c * SP + s] = 0.f;
            }
            return;
        }
    }
    float ph[3] = {0.f, 0.f, 0.f}, pl[3] = {0.f, 0.f, 0.f};
    if (active) {  // in the scatter, inactive lanes stay with their warp and add nothing
        const float *rf = rayf + (s / bd.nr) * kRayStride;
        const float t = ts[s];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            pos_two_float(rf[RF_O + a], t, rf[RF_D + a], ph[a], pl[a]);
    }
    const float2 *tab = reinterpret_cast<const float2 *>(od.theta);
    float2 *gtab = reinterpret_cast<float2 *>(od.grad);
#pragma unroll 2
    for (int l = part; l < L; l += PARTS) {
        const LevelDesc lv = od.lv[l];
        Corners cs;
        level_corners(lv, od.tmask, ph, pl, cs);
        PRENOM_CHECK_CORNERS(lv, od.tmask, cs, bd.status);
        if constexpr (!SCATTER) {
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
            XT[(2 * l) * SP + s] = e0;
            XT[(2 * l + 1) * SP + s] = e1;
        } else {
            const float g0 = active ? XT[(2 * l) * SP + s] : 0.f, g1 = active ? XT[(2 * l + 1) * SP + s] : 0.f;
            scatter_level_warp(gtab + lv.offset, active, cs, g0, g1, threadIdx.x & 31);
        }
    }
}

// ------------------------------------------------------------- compositing
// The ray's loss (Eq. 8-9, divided by the batch's ray count) and its
// gradients with respect to C-hat, D-hat and A (from the caller's upstream
// gradients in kRenderBwd mode).  ssum_total() gives the ray's sum of sigma,
// evaluated only for a background ray.
template <typename SsumFn>
__device__ __forceinline__ float ray_loss(const ObjDesc &od, const BatchDesc &bd, int gr, const float *rf,
                                          const float (&Cr)[3], float D, float A, SsumFn ssum_total, float (&gC)[3],
                                          float &gD, float &gA, bool &background)
{
    float loss = 0.f;
    background = false;
    if (bd.mode == kRenderBwd) {
        const float *up = bd.upstream + (size_t)gr * 5;
        gC[0] = up[0];
        gC[1] = up[1];
        gC[2] = up[2];
        gD = up[3];
        gA = up[4];
        return 0.f;
    }
    background = rf[RF_OBJ] < 0.5f;
    if (!background) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float e = Cr[c] - rf[RF_RGB + c];
            loss = fmaf(e, e, loss);
            gC[c] = 2.f * e;
        }
        const float ed = D - rf[RF_DEPTH];
        loss += od.lambda_d * fabsf(ed);
        gD = ed > 0.f ? od.lambda_d : (ed < 0.f ? -od.lambda_d : 0.f);
        gA = 0.f;
    } else {
        float dot = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float crd = rf[RF_CR + c];
            const float e = (Cr[c] + (1.f - A) * crd) - crd;
            loss = fmaf(e, e, loss);
            gC[c] = 2.f * e;
            dot = fmaf(2.f * e, crd, dot);
        }
        gD = 0.f;
        gA = -dot;
        loss = fmaf(od.lambda_sigma, ssum_total(), loss);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        gC[c] *= bd.inv_r;
    gD *= bd.inv_r;
    gA *= bd.inv_r;
    return loss * bd.inv_r;
}

__device__ __forceinline__ void group_bar(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Compositing (Eq. 7), loss and adjoint of one ray spread over G = ceil(nr / 32)
// warps, one sample per lane: warp g of the group holds samples 32 g .. 32 g + 31.
// Forward: tau_k = sigma_k delta_k, T_k = exp(-sum_{j<k} tau_j), w_k = T_k (1 - exp(-tau_k)).
// Adjoint with v_k = gC.c_k + gD t_k + gA:
//   dL/dsigma_k = delta_k (T_{k+1} v_k - sum_{j>k} w_j v_j).
// Writes dL/do (o = raw MLP outputs) into dOT; returns the ray's loss (train
// mode) on every warp of the group.  For G > 1 the warps meet through named
// barrier `bar` (G x 32 threads) and 8 floats per warp of `xs` (shared memory):
// the warp's sum of tau (slot 0), its partial sums of w c, w t, w and sigma
// (slots 1-6) and its sum of w v (slot 7), each combined in warp order.  For
// G = 1 nothing leaves the warp's registers.
template <int G>
__device__ __forceinline__ float composite_group(const ObjDesc &od, const BatchDesc &bd, int r, int gr,
                                                 const float *rf, const float *ts, const float *OT, float *dOT,
                                                 int SP, int lane, int wig, float *xs, int bar)
{
    const int nr = bd.nr;
    const int k = 32 * wig + lane;
    const bool valid = k < nr;
    const int s = r * nr + k;
    const float tf = rf[RF_TF];
    float o0 = 0.f, sig = 0.f, col[3] = {0.f, 0.f, 0.f}, tk = 0.f, dl = 0.f, tau = 0.f;
    if (valid) {
        o0 = OT[s];
        sig = expf(fminf(o0, 15.f));
        if (bd.out_sigma)
            bd.out_sigma[(size_t)gr * nr + k] = sig;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            col[c] = 1.f / (1.f + expf(-OT[(1 + c) * SP + s]));
        tk = ts[s];
        const float tnext = (k + 1 < nr) ? ts[s + 1] : tf;
        dl = tnext - tk;
        tau = sig * dl;
    }
    const float incl = warp_incl_scan(tau, lane);
    float excl = __shfl_up_sync(kFull, incl, 1);  // this warp's samples before this one
    if (lane == 0)
        excl = 0.f;
    if constexpr (G > 1) {
        if (lane == 31)
            xs[8 * wig] = incl;
        group_bar(bar, 32 * G);
    }
    float pref = 0.f;  // earlier warps' samples
#pragma unroll
    for (int g = 0; g < G - 1; ++g)
        if (g < wig)
            pref += xs[8 * g];
    const float T = expf(-(pref + excl));
    const float w = T * (-expm1f(-tau));
    float part[6] = {w * col[0], w * col[1], w * col[2], w * tk, w, sig};
#pragma unroll
    for (int i = 0; i < 6; ++i)
        part[i] = warp_sum(part[i]);
    float tot[6] = {part[0], part[1], part[2], part[3], part[4], part[5]};
    if constexpr (G > 1) {
        if (lane == 0)
#pragma unroll
            for (int i = 0; i < 6; ++i)
                xs[8 * wig + 1 + i] = part[i];
        group_bar(bar, 32 * G);
#pragma unroll
        for (int i = 0; i < 6; ++i)
            tot[i] = 0.f;
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int i = 0; i < 6; ++i)
                tot[i] += xs[8 * g + 1 + i];
    }
    const float Cr[3] = {tot[0], tot[1], tot[2]};
    const float D = tot[3], A = tot[4];
    if (bd.mode == kRender) {
        if (lane == 0 && wig == 0) {
            if (bd.out_rgb) {
                bd.out_rgb[(size_t)gr * 3 + 0] = Cr[0];
                bd.out_rgb[(size_t)gr * 3 + 1] = Cr[1];
                bd.out_rgb[(size_t)gr * 3 + 2] = Cr[2];
            }
            if (bd.out_depth)
                bd.out_depth[gr] = D;
            if (bd.out_acc)
                bd.out_acc[gr] = A;
        }
        return 0.f;
    }
    float gC[3], gD, gA;
    bool background;
    const float loss = ray_loss(od, bd, gr, rf, Cr, D, A, [&]() { return tot[5]; }, gC, gD, gA, background);
    // adjoint: suffix sums of w v over the ray
    const float v = fmaf(gC[0], col[0], fmaf(gC[1], col[1], fmaf(gC[2], col[2], fmaf(gD, tk, gA))));
    const float wv = w * v;
    const float sincl = warp_incl_suffix(wv, lane);
    if constexpr (G > 1) {
        if (lane == 0)
            xs[8 * wig + 7] = sincl;
        group_bar(bar, 32 * G);
    }
    float after = __shfl_down_sync(kFull, sincl, 1);  // later lanes of this warp
    if (lane == 31)
        after = 0.f;
#pragma unroll
    for (int g = G - 1; g > 0; --g)
        if (g > wig)
            after += xs[8 * g + 7];
    if (valid) {
        const float sig_reg = background ? od.lambda_sigma * bd.inv_r : 0.f;
        const float Tn = expf(-(pref + excl + tau));
        const float dsig = fmaf(dl, fmaf(Tn, v, -after), sig_reg);
        dOT[s] = (o0 < 15.f) ? dsig * sig : 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float dc = w * gC[c];
            dOT[(1 + c) * SP + s] = dc * col[c] * (1.f - col[c]);
        }
    }
    return loss;
}

// Compositing of a tile's nrt rays by all warps of the block: one warp per ray
// for rays of at most 32 samples, else G = ceil(nr / 32) warps per ray (G nrt
// <= 8 warps, as a tile holds 128 samples at most).  xs: 64 floats of scratch
// shared memory; named barriers 1 .. nrt.  Returns this thread's share of the
// tile's loss (each ray counted once, on one lane).
__device__ __forceinline__ float composite_tile(const ObjDesc &od, const BatchDesc &bd, int ray0, int nrt,
                                               const float *rayf, const float *ts, const float *OT, float *dOT,
                                               int SP, float *xs)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int G = (bd.nr + 31) >> 5;
    float lsum = 0.f;
    if (G == 1) {
        for (int r = warp; r < nrt; r += kThreads / 32) {
            const float lr = composite_group<1>(od, bd, r, ray0 + r, rayf + r * kRayStride, ts, OT, dOT, SP, lane, 0,
                                                nullptr, 0);
            if (lane == 0)
                lsum += lr;
        }
        return lsum;
    }
    const int r = warp / G, wig = warp % G;
    if (r >= nrt)
        return 0.f;
    float lr;
    switch (G) {
    case 2:
        lr = composite_group<2>(od, bd, r, ray0 + r, rayf + r * kRayStride, ts, OT, dOT, SP, lane, wig,
                                xs + 8 * G * r, 1 + r);
        break;
    case 3:
        lr = composite_group<3>(od, bd, r, ray0 + r, rayf + r * kRayStride, ts, OT, dOT, SP, lane, wig,
                                xs + 8 * G * r, 1 + r);
        break;
    default:
        lr = composite_group<4>(od, bd, r, ray0 + r, rayf + r * kRayStride, ts, OT, dOT, SP, lane, wig,
                                xs + 8 * G * r, 1 + r);
        break;
    }
    return (lane == 0 && wig == 0) ? lr : 0.f;
}

// Block-wide copy of a work item into shared memory (the inner loops then
// read the descriptors with broadcast shared loads).  Ends with a barrier.
__device__ __forceinline__ void stage_item(const WorkItem &src, WorkItem &dst)
{
    const int *s = reinterpret_cast<const int *>(&src);
    int *d = reinterpret_cast<int *>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(WorkItem) / sizeof(int)); i += blockDim.x)
        d[i] = s[i];
    __syncthreads();
}

// One ray's data into its kRayStride shared-memory floats, in four parts
// (f = 0 origin, 1 direction, 2 object targets, 3 background colour), so that
// four threads load a ray in parallel and a tile pays about one memory latency.
__device__ __forceinline__ void load_ray_fields(const BatchDesc &bd, int g, float *rf, int f)
{
    if (!PRENOM_BOUNDS_OK(g >= 0 && g < bd.n_rays, bd.status))
        return;
    {
        if (f < 2) {
            const float *src = (f == 0 ? bd.o : bd.d) + (size_t)g * 3;
#pragma unroll
            for (int a = 0; a < 3; ++a)
                rf[(f == 0 ? RF_O : RF_D) + a] = src[a];
        } else if (bd.mode == kTrain) {
            const bool obj = bd.is_obj[g] != 0;
            if (f == 2) {
                rf[RF_OBJ] = obj ? 1.f : 0.f;
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    rf[RF_RGB + a] = obj ? bd.rgb[(size_t)g * 3 + a] : 0.f;
                rf[RF_DEPTH] = obj ? bd.depth[g] : 0.f;
            } else if (!obj) {
                if (bd.c_rand) {
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        rf[RF_CR + a] = bd.c_rand[(size_t)g * 3 + a];
                } else {
                    const float3 c = philox_colour(bd.seed, bd.step, bd.obj_id, (uint32_t)g);
                    rf[RF_CR] = c.x;
                    rf[RF_CR + 1] = c.y;
                    rf[RF_CR + 2] = c.z;
                }
            }
        }
    }
}

__device__ __forceinline__ void load_ray_tile(const BatchDesc &bd, int ray0, int nrt, float *rayf)
{
    for (int i = threadIdx.x; i < nrt * 4; i += blockDim.x)
        load_ray_fields(bd, ray0 + (i >> 2), rayf + (i >> 2) * kRayStride, i & 3);
}

// Index of the work item owning launch-wide tile t (items sorted by tile_begin).
__device__ __forceinline__ int item_of_tile(const WorkItem *list, int n, int t)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (list[mid].tile_begin <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

}  // namespace prenom
