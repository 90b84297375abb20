// Mixed-precision fused training step (FP16 or BF16 MLP on the sm_100-family
// tensor cores, FP32 accumulation in tensor memory, FP32 master weights).
//
// Same tile walk as the FP32 kernel (sampling, encoding, compositing and the
// hash scatter are the FP32 code), but every MLP contraction is a tcgen05.mma
// issued by one thread:
//   forward   H_l   = relu(A_l W_l^T)       M = 128 samples, N = W, K = in
//   output    O     = H_last W_out^T         N = 16 (4 outputs, zero-padded)
//   backward  dH_l  = (dH_{l+1} W_{l+1})     masked by H_l > 0
//             dW_l += dH_l^T A_l             M = 64 (W zero-padded), K = 128 samples
//             dX    = dH_0 W_0               read by the scatter threads from TMEM
// Every 16-bit operand lives once in shared memory in the no-swizzle
// interleaved layout (8x8 core matrices of 128 contiguous bytes) and is used
// K-major or MN-major by the descriptors, so no transposed copies exist.  The
// weight gradients accumulate in tensor memory for the CTA's whole life and are
// flushed with one atomic pass at the end; dW_out (4 x W) too, as rows 0..3 of
// an M = 64 product, when its columns fit in the CTA's 256 (else it is summed
// on the CUDA cores while the tensor cores form dH of the last hidden layer).
// The backward gradients are multiplied by a loss scale before the 16-bit cast
// (FP16 dynamic range) and divided by it in FP32 on the way out.  Likewise an
// FP16 object's encoding is multiplied by a power of two 2^k before its cast, so
// that the small features and activations of a freshly initialised object stay
// FP16 normals: the layers have no biases and ReLU is positively homogeneous, so
// every hidden activation carries the same factor, which the output layer's
// FP32 products and every weight gradient divide out on the way out (dX does
// not carry it).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fused_fp32.cuh"

namespace prenom {

template <bool BF16>
struct Half;

template <>
struct Half<true> {
    static constexpr uint32_t fmt = 1;  // instruction-descriptor operand format
    static __device__ __forceinline__ uint16_t bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
    static __device__ __forceinline__ float value(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }
    static __device__ __forceinline__ bool finite(uint16_t b) { return (b & 0x7F80u) != 0x7F80u; }
    // two values in one conversion, a in the low half
    static __device__ __forceinline__ uint32_t pack2(float a, float b)
    {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    static constexpr float kRoundsToInf = 3.3961e38f;  // |x| from here on rounds to infinity
};

template <>
struct Half<false> {
    static constexpr uint32_t fmt = 0;
    static __device__ __forceinline__ uint16_t bits(float x) { return __half_as_ushort(__float2half_rn(x)); }
    static __device__ __forceinline__ float value(uint16_t b) { return __half2float(__ushort_as_half(b)); }
    static __device__ __forceinline__ bool finite(uint16_t b) { return (b & 0x7C00u) != 0x7C00u; }
    static __device__ __forceinline__ uint32_t pack2(float a, float b)
    {
        const __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<const uint32_t *>(&h);
    }
    static constexpr float kRoundsToInf = 65520.f;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (r, c) of a rows x cols 16-bit matrix in the
// interleaved layout: core matrix (r/8, c/8) at (r/8)*(cols/8)*128 + (c/8)*128,
// row r%8 of a core at 16 B, element c%8 at 2 B.
__device__ __forceinline__ int il_off(int r, int c, int cols)
{
    return ((r >> 3) * (cols >> 3) + (c >> 3)) * 128 + (r & 7) * 16 + (c & 7) * 2;
}

// An MMA operand: a stored matrix viewed K-major (its rows are M or N) or
// MN-major (its rows are K).  kstr / mnstr: byte distance of adjacent core
// matrices along K and along M (or N).
struct Operand {
    uint32_t addr, kstr, mnstr, mn_major;
};

__device__ __forceinline__ Operand kmajor(const void *p, int cols)
{
    return Operand{smem_addr(p), 128u, (uint32_t)(cols >> 3) * 128u, 0u};
}

__device__ __forceinline__ Operand mnmajor(const void *p, int cols)
{
    return Operand{smem_addr(p), (uint32_t)(cols >> 3) * 128u, 128u, 1u};
}

// Shared-memory matrix descriptor: start, leading (K-direction) and stride
// (M/N-direction) byte offsets in 16-byte units, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, 16-bit A and B of the
// given format, major-ness of A and B, N >> 3 and M >> 4.
__device__ __forceinline__ uint32_t mma_idesc(uint32_t fmt, int M, int N, uint32_t a_mn, uint32_t b_mn)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | (a_mn << 15) | (b_mn << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// D (+)= A * B^T over K (a multiple of 16, known at compile time), issued by
// the calling thread.  The descriptors are built once; each further K = 16
// slice only advances their start-address field (14 bits of address / 16: a
// shared-memory address below 256 KB never carries out of it), so the single
// issuing thread spends a few cycles per MMA instead of a dependent chain of
// 64-bit shifts and masks.
// kslices (<= K / 16) issues only the first slices: a weight-gradient product
// over a tile's samples stops after its last filled sample (rows past it are
// zero in both operands, so the result is the same).
template <int K>
__device__ __forceinline__ void mma_gemm(uint32_t d_tmem, const Operand &a, const Operand &b, uint32_t idesc,
                                         bool accumulate, int kslices = K / 16)
{
    static_assert(K % 16 == 0 && K > 0, "K is a multiple of 16");
    const uint64_t ad0 = smem_desc(a.addr, a.kstr, a.mnstr);
    const uint64_t bd0 = smem_desc(b.addr, b.kstr, b.mnstr);
    const uint64_t astep = (uint64_t)((2u * a.kstr) >> 4), bstep = (uint64_t)((2u * b.kstr) >> 4);
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks) {
        if (ks >= kslices)
            break;
        const uint64_t ad = ad0 + (uint64_t)ks * astep;
        const uint64_t bd = bd0 + (uint64_t)ks * bstep;
        const uint32_t acc = (accumulate || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_addr(mbar)));
}

// Bounded poll of the mbarrier phase by this thread alone (no barrier): false
// (and status set) when it gave up.  Every caller combines the answers of
// all threads at its next tc_sync_and, so that no thread leaves a loop alone.
__device__ __forceinline__ bool mbar_poll(uint64_t *mbar, uint32_t parity, int32_t *status)
{
    uint32_t done = 0;
    for (int it = 0; it < (1 << 24) && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_addr(mbar)), "r"(parity));
    }
    if (!done && status)
        atomicOr(status, kStatusWait);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return done != 0;
}

// tc_sync that also returns, to every thread, whether all threads passed `ok`.
__device__ __forceinline__ bool tc_sync_and(bool ok)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    const bool all = __syncthreads_and(ok) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return all;
}

__device__ __forceinline__ void tc_sync()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i)
        v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8])
{
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i)
        v[i] = __uint_as_float(r[i]);
}

// N (8, 16 or 32) consecutive FP32 columns of this thread's TMEM lane: every
// 8-column load is issued before the one wait, whose register operands tie
// the loaded values to it so that no use moves above it.
template <int N>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float (&v)[N])
{
    static_assert(N == 8 || N == 16 || N == 32, "columns");
    uint32_t r[N];
#pragma unroll
    for (int q = 0; q < N / 8; ++q)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[8 * q]), "=r"(r[8 * q + 1]), "=r"(r[8 * q + 2]), "=r"(r[8 * q + 3]),
                       "=r"(r[8 * q + 4]), "=r"(r[8 * q + 5]), "=r"(r[8 * q + 6]), "=r"(r[8 * q + 7])
                     : "r"(taddr + 8 * q));
    if constexpr (N == 8) {
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
                     :
                     : "memory");
    } else if constexpr (N == 16) {
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                       "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                       "+r"(r[15])
                     :
                     : "memory");
    } else {
        asm volatile("tcgen05.wait::ld.sync.aligned;"
                     : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                       "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                       "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                       "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                       "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                     :
                     : "memory");
    }
#pragma unroll
    for (int i = 0; i < N; ++i)
        v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4])
{
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 4; ++i)
        v[i] = __uint_as_float(r[i]);
}

constexpr int kTcTile = 128;       // samples per tile = MMA M
constexpr int kTcCols = 256;       // most TMEM columns a CTA allocates
constexpr int kDaCols = 64;        // columns of the dH buffer (dW MMAs use M = 64)

// dW_out (4 x W) on the tensor cores, at dw_col(H): for W = 64 as its transpose
// dW_out^T = H_{H-1}^T dO (M = 64 = W, N = 16: dO's 16 zero-padded columns, so 16
// TMEM columns and the plain 16-column dO buffer), for W < 64 as rows 0..3 of an
// M = 64 accumulator of W columns (dO widened to 64 columns); when its columns do
// not fit after the hidden layers' dW (for the launch's deepest MLP) it is summed
// on the CUDA cores.
template <int W>
__host__ __device__ __forceinline__ constexpr bool tc_dwo_transposed()
{
    return W == kDaCols;
}

// TMEM columns of R0, the region that holds in turn a forward layer (W), the
// output layer (16), a backward product (W) and dX (the padded encoding width).
template <int W, int IN>
__host__ __device__ __forceinline__ constexpr int tc_r0()
{
    return W > (IN < 16 ? 16 : IN) ? W : (IN < 16 ? 16 : IN);
}

template <int W, int IN>
__host__ __device__ __forceinline__ constexpr bool tc_dw_out(int H)
{
    return tc_r0<W, IN>() + (IN < 16 ? 16 : IN) + (H - 1) * W + (tc_dwo_transposed<W>() ? 16 : W) <= kTcCols;
}

template <int W, int IN>
struct TcLayout {
    static constexpr int INP = IN < 16 ? 16 : IN;  // encoding width padded to the MMA N/K quantum
    static constexpr int SP = kTcTile + 4;
    // byte sizes of the 16-bit matrices
    static constexpr int w0 = W * INP * 2, wh = W * W * 2, wo = 16 * W * 2;
    static constexpr int xa = kTcTile * INP * 2, ha = kTcTile * W * 2, da = kTcTile * kDaCols * 2;
    // dO: 4 of 16 columns (the K of the dH product and the N of the transposed
    // dW_out product), or of 64 when the M = 64 dW_out product reads it
    static __host__ __device__ int doa_cols(int H, bool split)
    {
        return split && tc_dw_out<W, IN>(H) && !tc_dwo_transposed<W>() ? kDaCols : 16;
    }
    // floats of the per-warp scratch: the sampler's CDFs, or in split mode (no
    // sampler in this kernel) only the compositing's exchange, 8 per warp
    static __host__ __device__ int scratch_floats(bool split) { return split ? 64 : 8 * (kMaxNc + 1); }
    static __host__ __device__ size_t bytes(int H, bool split)
    {
        size_t b = (size_t)w0 + (size_t)(H - 1) * wh + wo + xa + (size_t)H * ha + da;
        b += (size_t)kTcTile * doa_cols(H, split) * 2;
        b += sizeof(float) * (8 * SP + SP + (size_t)(kTcTile / kMinNr) * kRayStride + scratch_floats(split));
        return b + 64;  // TMEM slot and mbarrier
    }
};

// TMEM column of each accumulator region: R0 (tc_r0 columns) holds the
// current forward layer, the output layer, then the current backward product
// and dX; the dW accumulators follow (M = 64 layout: row m in lane
// 32*(m/16) + m%16).
template <int W, int IN>
__host__ __device__ __forceinline__ uint32_t dw_col(int layer)
{
    constexpr int INP = TcLayout<W, IN>::INP;
    constexpr int R0 = tc_r0<W, IN>();
    return layer == 0 ? (uint32_t)R0 : (uint32_t)(R0 + INP + (layer - 1) * W);
}

// TMEM columns a CTA allocates for a launch whose deepest MLP has H hidden
// layers: R0, the dW accumulators and, where it is formed on the tensor cores,
// dW_out, rounded up to a power of two (at least 32).  A width-16 or width-32
// MLP of at most two hidden layers needs 128, so up to four CTAs share an SM's
// 512 columns; a width-64 MLP needs 256.
template <int W, int IN>
__host__ __device__ __forceinline__ int tc_cols(int H, bool split)
{
    const int need = (int)dw_col<W, IN>(H) + ((split && tc_dw_out<W, IN>(H)) ? (tc_dwo_transposed<W>() ? 16 : W) : 0);
    int cols = 32;
    while (cols < need)
        cols *= 2;
    return cols;
}

// Resident CTAs per SM that the split form's MLP kernel budgets its registers
// for: three for widths up to 32 (80 registers a thread), two otherwise.
template <int W, bool SPLIT>
__host__ __device__ __forceinline__ constexpr int tc_min_blocks()
{
    return (SPLIT && W <= 32) ? 3 : 2;
}


// 16-bit weights of one object into the interleaved buffers (their padding
// rows and columns were cleared once at kernel start and are never written).
template <int W, int IN, bool BF16>
__device__ __forceinline__ void tc_load_object(const ObjDesc &od, unsigned char *Wt0, unsigned char *WtH,
                                               unsigned char *WtO)
{
    using Hf = Half<BF16>;
    constexpr int INP = TcLayout<W, IN>::INP;
    const int H = od.H;
    const float *th = od.theta + od.mlp_off;
    for (int i = threadIdx.x; i < W * IN; i += kThreads) {
        const int o = i / IN, c = i % IN;
        *reinterpret_cast<uint16_t *>(Wt0 + il_off(o, c, INP)) = Hf::bits(th[i]);
    }
    for (int l = 1; l < H; ++l)
        for (int i = threadIdx.x; i < W * W; i += kThreads) {
            const int o = i / W, c = i % W;
            *reinterpret_cast<uint16_t *>(WtH + (l - 1) * TcLayout<W, IN>::wh + il_off(o, c, W)) =
                Hf::bits(th[IN * W + (l - 1) * W * W + i]);
        }
    for (int i = threadIdx.x; i < 4 * W; i += kThreads) {
        const int o = i / W, c = i % W;
        *reinterpret_cast<uint16_t *>(WtO + il_off(o, c, W)) = Hf::bits(th[IN * W + (H - 1) * W * W + i]);
    }
}

// Loss, dW_out (CUDA-core sums) and the TMEM weight-gradient accumulators of
// the CTA into the object (all threads call it; M = 64 accumulator layout:
// warp quadrant q holds rows 16q .. 16q+15 in its lanes 0..15).
template <int W, int IN>
__device__ __forceinline__ void tc_flush_object(const ObjDesc &od, const BatchDesc &bd, uint32_t lane_base,
                                                bool have_dw, bool tc_dwo, float (&dwo_acc)[8], float &loss_acc,
                                                float inv_scale, float inv_enc)
{
    constexpr int INP = TcLayout<W, IN>::INP;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int quad = warp & 3, half = warp >> 2;
    if (lane == 0 && bd.mode == kTrain && loss_acc != 0.f)
        red_add_f(bd.loss, loss_acc);
    loss_acc = 0.f;
    if (bd.mode == kRender)
        return;
    const int H = od.H;
    float *gw = od.grad + od.mlp_off;
    if (!tc_dwo) {  // dW_out from the CUDA cores: slice 0 of each (output, 8-column) group holds its sums
        constexpr int SL = kThreads / (W / 2);
        const int pair = tid / SL;
        const int o = pair / (W / 8), i0 = (pair % (W / 8)) * 8;
        if (tid % SL == 0) {  // 16-byte reductions: the 304-way contention per address is per request
            float4 *p = reinterpret_cast<float4 *>(gw + IN * W + (H - 1) * W * W + o * W + i0);
            const float f = inv_scale * inv_enc;  // dO times the scaled activations
            red_add_f4(p, dwo_acc[0] * f, dwo_acc[1] * f, dwo_acc[2] * f, dwo_acc[3] * f);
            red_add_f4(p + 1, dwo_acc[4] * f, dwo_acc[5] * f, dwo_acc[6] * f, dwo_acc[7] * f);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
            dwo_acc[j] = 0.f;
    }
    if (!have_dw)
        return;
    if (tc_dwo && tc_dwo_transposed<W>()) {  // dW_out^T: row i of TMEM holds dW_out[0..3][i]
        if (half == 0) {
            float v[8];
            tmem_ld8(lane_base + dw_col<W, IN>(H), v);
            const int i = 16 * quad + lane;
            if (lane < 16) {
                float *dst = gw + IN * W + (H - 1) * W * W + i;
                const float f = inv_scale * inv_enc;
#pragma unroll
                for (int o = 0; o < 4; ++o)
                    red_add_f(dst + o * W, v[o] * f);
            }
        }
    }
    for (int l = 0; l < H + (tc_dwo && !tc_dwo_transposed<W>() ? 1 : 0); ++l) {  // layer H: dW_out, 4 rows
        const int ncol = l == 0 ? INP : W;
        const int nin = l == 0 ? IN : W;
        const int nrow = l == H ? 4 : W;
        float *dst = gw + (l == 0 ? 0 : IN * W + (l - 1) * W * W);
        const float f = inv_scale * inv_enc;  // every dW was formed from scaled inputs of its layer
        for (int c0 = half * 8; c0 < ncol; c0 += 16) {
            float v[8];
            tmem_ld8(lane_base + dw_col<W, IN>(l) + c0, v);
            const int row = 16 * quad + lane;
            if (lane < 16 && row < nrow && c0 < nin) {  // nin and c0 are multiples of 8: two aligned quads
                float4 *p = reinterpret_cast<float4 *>(dst + row * nin + c0);
                red_add_f4(p, v[0] * f, v[1] * f, v[2] * f, v[3] * f);
                red_add_f4(p + 1, v[4] * f, v[5] * f, v[6] * f, v[7] * f);
            }
        }
    }
}

// SPLIT: the split form's MLP kernel (sampling, encoding and the scatter run in
// kernels of their own), instantiated apart from the fused kernel so that its
// code holds only what it runs (fewer instruction-fetch stalls); it must match
// wl.split, and each item's hand-over buffers must be present.
template <int W, int IN, bool BF16, bool SPLIT>
__global__ void __launch_bounds__(kThreads, tc_min_blocks<W, SPLIT>())
    fused_tc_kernel(const __grid_constant__ WorkItem one, const WorkList wl)
{
    using L = TcLayout<W, IN>;
    using Hf = Half<BF16>;
    constexpr int INP = L::INP;
    constexpr int SP = L::SP;
    constexpr int MAXR = kTcTile / kMinNr;
    constexpr int NL = IN / 2;  // levels (F = 2)
    extern __shared__ __align__(128) unsigned char smc[];
    const WorkItem *list = wl.items ? wl.items : &one;
    const int n_items = wl.items ? wl.n_items : 1;
    const int total = wl.items ? wl.total_tiles : one.bd.n_tiles;
    const int hmax = wl.items ? wl.hmax : one.od.H;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int quad = warp & 3, half = warp >> 2;
    const int srow = 32 * quad + lane;  // TMEM lane = sample row of this thread

    unsigned char *Wt0 = smc;
    unsigned char *WtH = Wt0 + L::w0;                 // layers 1..H-1
    unsigned char *WtO = WtH + (hmax - 1) * L::wh;
    unsigned char *XA = WtO + L::wo;
    unsigned char *HA = XA + L::xa;                   // H buffers of ha bytes
    unsigned char *DA = HA + hmax * L::ha;
    unsigned char *DOA = DA + L::da;
    // dW_out on the tensor cores, for every object of the launch (H <= hmax): only in
    // split mode, where the kernel gathers nothing and the wider dO buffer does not
    // take L1 cache away from the hash gathers.  Its columns fit beside the hidden
    // layers' dW for every width and depth the library accepts, so the choice is the
    // variant's (the CUDA-core dW_out path is compiled into the fused variant only)
    static_assert(!SPLIT || tc_dw_out<W, IN>(kMaxHidden), "split mode forms dW_out on the tensor cores");
    constexpr bool tc_dwo = SPLIT;
    const int doa_cols = L::doa_cols(hmax, SPLIT);
    float *OT = reinterpret_cast<float *>(DOA + kTcTile * doa_cols * 2);  // [4][SP] raw outputs
    float *dOT = OT + 4 * SP;                         // [4][SP] dL/d(raw outputs), unscaled
    float *ts = dOT + 4 * SP;
    float *rayf = ts + SP;
    float *cdfs = rayf + MAXR * kRayStride;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(cdfs + L::scratch_floats(SPLIT));
    uint64_t *mbar = reinterpret_cast<uint64_t *>(tmem_slot + 2);

    // buffers with padding that is never written again: W_0 (columns IN..INP),
    // W_out (rows 4..15), DA (columns W..63), dO (columns 4..15)
    for (int i = tid; i < L::w0 / 4; i += kThreads)
        reinterpret_cast<uint32_t *>(Wt0)[i] = 0u;
    for (int i = tid; i < L::wo / 4; i += kThreads)
        reinterpret_cast<uint32_t *>(WtO)[i] = 0u;
    for (int i = tid; i < L::da / 4; i += kThreads)
        reinterpret_cast<uint32_t *>(DA)[i] = 0u;
    for (int i = tid; i < kTcTile * doa_cols / 2; i += kThreads)
        reinterpret_cast<uint32_t *>(DOA)[i] = 0u;
    __syncthreads();
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const uint32_t ncols = (uint32_t)tc_cols<W, IN>(hmax, SPLIT);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quad) << 16);

    const uint32_t id_fwd = mma_idesc(Hf::fmt, 128, W, 0, 0);
    const uint32_t id_out = mma_idesc(Hf::fmt, 128, 16, 0, 0);
    const uint32_t id_dh = mma_idesc(Hf::fmt, 128, W, 0, 1);
    const uint32_t id_dx = mma_idesc(Hf::fmt, 128, INP, 0, 1);
    const uint32_t id_dw = mma_idesc(Hf::fmt, 64, W, 1, 1);
    const uint32_t id_dwo_t = mma_idesc(Hf::fmt, 64, 16, 1, 1);  // dW_out^T (W = 64)
    const uint32_t id_dw0 = mma_idesc(Hf::fmt, 64, INP, 1, 1);

    uint32_t parity = 0;
    bool ok = true;
    bool first_dw = true;
    float dwo_acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // dW_out entries of this thread's group
    float loss_acc = 0.f;
    float scale = 1.f, inv_scale = 1.f;
    float enc = 1.f, inv_enc = 1.f;  // FP16: power of two applied to the encoding before its cast

    __shared__ __align__(16) WorkItem cur;  // the item being processed
    const int per = (total + (int)gridDim.x - 1) / (int)gridDim.x;
    const int t0 = (int)blockIdx.x * per, t1 = min(total, t0 + per);
    int k = -1;
    // split mode: the next tile's copy-in, loaded into registers during this
    // tile's backward pass (image chunks, ray data, depths of two passes each)
    constexpr int kChunks = kTcTile * INP * 2 / 16;
    static_assert(kChunks <= 2 * kThreads && kTcRayMax * kRayStride <= 2 * kThreads && kTcTile <= kThreads,
                  "two registers per thread carry a tile");
    uint4 px0 = make_uint4(0u, 0u, 0u, 0u), px1 = px0;
    float pr0 = 0.f, pr1 = 0.f, pt0 = 0.f;
    int pre_t = -1;
    for (int t = t0; t < t1 && ok; ++t) {
        int nk = k < 0 ? item_of_tile(list, n_items, t) : k;
        while (nk + 1 < n_items && list[nk + 1].tile_begin <= t)
            ++nk;
        if (nk != k) {  // entering another object: flush the previous one, load this one
            if (k >= 0)
                tc_flush_object<W, IN>(cur.od, cur.bd, lane_base, !first_dw, tc_dwo, dwo_acc, loss_acc, inv_scale,
                                       inv_enc);
            __syncthreads();
            stage_item(list[nk], cur);
            tc_load_object<W, IN, BF16>(cur.od, Wt0, WtH, WtO);
            k = nk;
            first_dw = true;
            const BatchDesc &nb = cur.bd;
            scale = (nb.mode != kRender && nb.loss_scale) ? *nb.loss_scale : 1.f;
            inv_scale = 1.f / scale;
            enc = nb.enc_scale ? *nb.enc_scale : 1.f;
            inv_enc = 1.f / enc;  // exact: enc is a power of two
            tc_sync();
        }
        const ObjDesc &od = cur.od;
        const BatchDesc &bd = cur.bd;
        const int H = od.H;
        const bool train = bd.mode != kRender;
        const int nr = bd.nr, NR = bd.rays_per_tile;
        const int tile = t - cur.tile_begin;
        const int ray0 = tile * NR;
        const int nrt = min(NR, bd.n_rays - ray0);
        const int ns = nrt * nr;
        const int kdw = (ns + 15) >> 4;  // 16-sample slices of the weight-gradient products
        // ---- ray data and sampling (FP32, shared with the FP32 kernel)
        constexpr bool split = SPLIT;  // sampling, encoding and scatter run in kernels of their own
        if (SPLIT != (bd.sp_x != nullptr)) {  // a work list at odds with the variant: nothing is touched
            if (tid == 0 && bd.status)
                atomicOr(bd.status, kStatusWait);
            break;  // block-uniform (cur is shared)
        }
        if (split && pre_t == t) {  // prefetched during the previous tile
            if (tid < kChunks)
                reinterpret_cast<uint4 *>(XA)[tid] = px0;
            if (tid + kThreads < kChunks)
                reinterpret_cast<uint4 *>(XA)[tid + kThreads] = px1;
            if (tid < nrt * kRayStride)
                rayf[tid] = pr0;
            if (tid + kThreads < nrt * kRayStride)
                rayf[tid + kThreads] = pr1;
            if (tid < ns)
                ts[tid] = pt0;
            if (tid < kTcTile && tid >= ns)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    dOT[c * SP + tid] = 0.f;
        } else if (split) {
            // the tile's ray data, sample depths and encoding image from the sampling-encoding
            // kernel, in one pass (rows of the image past the samples zeroed)
            const float *rsrc = bd.sp_rays + (size_t)tile * kSplitRayFloats;
            for (int i = tid; i < nrt * kRayStride; i += kThreads)
                rayf[i] = rsrc[i];
            for (int i = tid; i < ns; i += kThreads)
                ts[i] = bd.sp_t[(size_t)ray0 * nr + i];
            const uint4 *src = bd.sp_x + (size_t)tile * (kSplitXBytes / 16);
            for (int i = tid; i < kTcTile * INP * 2 / 16; i += kThreads) {
                const int row = ((i >> 3) / (INP >> 3)) * 8 + (i & 7);
                reinterpret_cast<uint4 *>(XA)[i] = row < ns ? __ldcs(src + i) : make_uint4(0u, 0u, 0u, 0u);
            }
            if (tid < kTcTile && tid >= ns)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    dOT[c * SP + tid] = 0.f;
        } else {
            load_ray_tile(bd, ray0, nrt, rayf);
            __syncthreads();
            for (int r = warp; r < nrt; r += kThreads / 32)
                sample_ray_warp(od, bd, r, ray0 + r, rayf + r * kRayStride, ts, cdfs + warp * (kMaxNc + 1), lane);
            __syncthreads();
            // ---- encoding -> XA (16-bit, interleaved [128][INP])
            const int s = tid % kTcTile, part = tid / kTcTile;
            if (s >= ns) {
                for (int l = part; l < INP / 2; l += 2)
                    *reinterpret_cast<uint32_t *>(XA + il_off(s, 2 * l, INP)) = 0u;
                if (part == 0)
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        dOT[c * SP + s] = 0.f;
            } else {
                const int r = s / nr;
                const float *rf = rayf + r * kRayStride;
                const float t = ts[s];
                float ph[3], pl[3];
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    pos_two_float(rf[RF_O + a], t, rf[RF_D + a], ph[a], pl[a]);
                const float2 *tab = reinterpret_cast<const float2 *>(od.theta);
#pragma unroll 2
                for (int l = part; l < NL; l += 2) {
                    const LevelDesc lv = od.lv[l];
                    Corners cs;
                    level_corners(lv, od.tmask, ph, pl, cs);
                    PRENOM_CHECK_CORNERS(lv, od.tmask, cs, bd.status);
                    float2 f[8];
                    if (od.feat16) {  // the tables' BF16 copy
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
                    *reinterpret_cast<uint32_t *>(XA + il_off(s, 2 * l, INP)) =
                        Hf::pack2(e0 * enc, e1 * enc);
                }
                for (int l = NL + part; l < INP / 2; l += 2)  // zero padding of a narrow encoding
                    *reinterpret_cast<uint32_t *>(XA + il_off(s, 2 * l, INP)) = 0u;
            }
        }
        tc_sync();
        // ---- MLP forward on the tensor cores
        for (int l = 0; l < H && ok; ++l) {
            if (tid == 0) {
                const Operand a = l == 0 ? kmajor(XA, INP) : kmajor(HA + (l - 1) * L::ha, W);
                const Operand b = l == 0 ? kmajor(Wt0, INP) : kmajor(WtH + (l - 1) * L::wh, W);
                if (l == 0)
                    mma_gemm<INP>(tmem, a, b, id_fwd, false);
                else
                    mma_gemm<W>(tmem, a, b, id_fwd, false);
                mma_commit(mbar);
            }
            const bool done = mbar_poll(mbar, parity, bd.status);
            parity ^= 1u;
            // epilogue: relu -> 16-bit -> HA[l]; warp half h takes columns [h W/2, (h+1) W/2)
            // (the activations keep the encoding's scale: the layers are linear up to ReLU)
            {
                float v[W / 2];
                tmem_ld_cols<W / 2>(lane_base + half * (W / 2), v);
#pragma unroll
                for (int c0 = 0; c0 < W / 2; c0 += 8) {
                    const int col = half * (W / 2) + c0;
                    uint4 pk;
                    pk.x = Hf::pack2(fmaxf(v[c0], 0.f), fmaxf(v[c0 + 1], 0.f));
                    pk.y = Hf::pack2(fmaxf(v[c0 + 2], 0.f), fmaxf(v[c0 + 3], 0.f));
                    pk.z = Hf::pack2(fmaxf(v[c0 + 4], 0.f), fmaxf(v[c0 + 5], 0.f));
                    pk.w = Hf::pack2(fmaxf(v[c0 + 6], 0.f), fmaxf(v[c0 + 7], 0.f));
                    *reinterpret_cast<uint4 *>(HA + l * L::ha + il_off(srow, col, W)) = pk;
                }
            }
            ok = tc_sync_and(done);
        }
        if (!ok)
            break;
        if (tid == 0) {
            mma_gemm<W>(tmem, kmajor(HA + (H - 1) * L::ha, W), kmajor(WtO, W), id_out, false);
            mma_commit(mbar);
        }
        {
            const bool done = mbar_poll(mbar, parity, bd.status);
            parity ^= 1u;
            if (half == 0) {
                float v[4];
                tmem_ld4(lane_base, v);
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    OT[c * SP + srow] = v[c] * inv_enc;  // the raw outputs without the encoding's scale
            }
            ok = tc_sync_and(done);
        }
        if (!ok)
            break;
        pre_t = -1;
        if (split && t + 1 < t1 && tile + 1 < bd.n_tiles) {  // the next tile of this item: issue its loads now,
            // so that they are in flight through the compositing and the backward pass
            const int tile2 = tile + 1, ray02 = tile2 * NR;
            const int ns2 = min(NR, bd.n_rays - ray02) * nr, nr2 = min(NR, bd.n_rays - ray02) * kRayStride;
            const uint4 *src = bd.sp_x + (size_t)tile2 * (kSplitXBytes / 16);
            const uint4 z = make_uint4(0u, 0u, 0u, 0u);
            const int i1 = tid + kThreads;
            px0 = tid < kChunks && ((tid >> 3) / (INP >> 3)) * 8 + (tid & 7) < ns2 ? __ldcs(src + tid) : z;
            px1 = i1 < kChunks && ((i1 >> 3) / (INP >> 3)) * 8 + (i1 & 7) < ns2 ? __ldcs(src + i1) : z;
            const float *rsrc = bd.sp_rays + (size_t)tile2 * kSplitRayFloats;
            pr0 = tid < nr2 ? rsrc[tid] : 0.f;
            pr1 = i1 < nr2 ? rsrc[i1] : 0.f;
            pt0 = tid < ns2 ? bd.sp_t[(size_t)ray02 * nr + tid] : 0.f;
            pre_t = t + 1;
        }
        // ---- compositing, loss and its adjoint (FP32)
        // (the sampler's CDF scratch serves as the compositing's exchange buffer)
        loss_acc += composite_tile(od, bd, ray0, nrt, rayf, ts, OT, dOT, SP, cdfs);
        __syncthreads();
        if (!train)
            continue;
        // ---- scaled 16-bit dL/dO (dW_out is summed during the first backward product)
        if (tid < kTcTile) {
            uint32_t lo = (uint32_t)Hf::bits(dOT[tid] * scale) | ((uint32_t)Hf::bits(dOT[SP + tid] * scale) << 16);
            uint32_t hi = (uint32_t)Hf::bits(dOT[2 * SP + tid] * scale) |
                          ((uint32_t)Hf::bits(dOT[3 * SP + tid] * scale) << 16);
            *reinterpret_cast<uint2 *>(DOA + il_off(tid, 0, doa_cols)) = make_uint2(lo, hi);
            if (!(Hf::finite(lo & 0xFFFFu) && Hf::finite(lo >> 16) && Hf::finite(hi & 0xFFFFu) &&
                  Hf::finite(hi >> 16)) && bd.overflow)
                atomicExch(bd.overflow, 1);
        }
        tc_sync();
        // ---- backward through the hidden layers
        for (int l = H - 1; l >= 0 && ok; --l) {
            // dH_l = dOut_{l+1} W_{l+1}: for l = H-1 from the output layer
            if (tid == 0) {
                if (l == H - 1)
                    mma_gemm<16>(tmem, kmajor(DOA, doa_cols), mnmajor(WtO, W), id_dh, false);
                else
                    mma_gemm<W>(tmem, kmajor(DA, kDaCols), mnmajor(WtH + l * L::wh, W), id_dh, false);
                mma_commit(mbar);
                if (l == H - 1 && tc_dwo) {  // dW_out (a later commit covers it)
                    if constexpr (tc_dwo_transposed<W>())  // dW_out^T += H_{H-1}^T dO
                        mma_gemm<kTcTile>(tmem + dw_col<W, IN>(H), mnmajor(HA + (H - 1) * L::ha, W),
                                          mnmajor(DOA, 16), id_dwo_t, !first_dw, kdw);
                    else  // dW_out += dO^T H_{H-1}, rows 0..3 of M = 64
                        mma_gemm<kTcTile>(tmem + dw_col<W, IN>(H), mnmajor(DOA, kDaCols),
                                          mnmajor(HA + (H - 1) * L::ha, W), id_dw, !first_dw, kdw);
                }
            }
            if (l == H - 1 && !tc_dwo) {
                // dW_out[o][i0..i0+7] on the CUDA cores while the tensor cores form dH_{H-1}:
                // each thread sums an interleaved slice of the tile's samples (conflict-free
                // 16-byte rows of H), the slices meet by shuffles
                constexpr int SL = kThreads / (W / 2);  // slices per output group (8, 16, 32 for W = 64, 32, 16)
                const int pair = tid / SL, slice = tid % SL;
                const int o = pair / (W / 8), i0 = (pair % (W / 8)) * 8;
                const unsigned char *hl = HA + (H - 1) * L::ha;
                float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
                for (int k = 0; k < kTcTile / SL; ++k) {
                    if (k * SL >= ns)  // the tile's empty rows add nothing
                        break;
                    const int s = k * SL + slice;
                    // the same 16-bit dO (scaled) the tensor-core form multiplies
                    const float d = Hf::value(Hf::bits(dOT[o * SP + s] * scale));
                    const uint4 hv = *reinterpret_cast<const uint4 *>(hl + il_off(s, i0, W));
                    const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        acc[2 * j] = fmaf(d, Hf::value((uint16_t)(hw[j] & 0xFFFFu)), acc[2 * j]);
                        acc[2 * j + 1] = fmaf(d, Hf::value((uint16_t)(hw[j] >> 16)), acc[2 * j + 1]);
                    }
                }
#pragma unroll
                for (int off = SL / 2; off > 0; off >>= 1)
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        acc[j] += __shfl_xor_sync(kFull, acc[j], off);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    dwo_acc[j] += acc[j];  // meaningful in slice 0 of each group
            }
            const bool done = mbar_poll(mbar, parity, bd.status);
            parity ^= 1u;
            // epilogue: mask by H_l > 0 -> 16-bit -> DA (columns [0, W))
            const unsigned char *hl = HA + l * L::ha;
            float vb[W / 2];
            tmem_ld_cols<W / 2>(lane_base + half * (W / 2), vb);
            // an H entry is > 0 iff its 16-bit pattern is neither +0 nor -0 (the ReLU output
            // is never negative or NaN); a masked value overflows the 16-bit format iff its
            // magnitude reaches the rounding threshold to infinity, and a NaN shows in the
            // sum of magnitudes (fmaxf would drop it)
            float amax = 0.f, asum = 0.f;
#pragma unroll
            for (int c0 = 0; c0 < W / 2; c0 += 8) {
                const int col = half * (W / 2) + c0;
                const float *v = vb + c0;
                const uint4 hv = *reinterpret_cast<const uint4 *>(hl + il_off(srow, col, W));
                const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
                uint32_t pk[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float a = (hw[j] & 0x7FFFu) ? v[2 * j] : 0.f;
                    const float b = (hw[j] & 0x7FFF0000u) ? v[2 * j + 1] : 0.f;
                    amax = fmaxf(amax, fmaxf(fabsf(a), fabsf(b)));
                    asum += fabsf(a) + fabsf(b);
                    pk[j] = Hf::pack2(a, b);
                }
                *reinterpret_cast<uint4 *>(DA + il_off(srow, col, kDaCols)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
            if ((!(amax < Hf::kRoundsToInf) || asum != asum) && bd.overflow)
                atomicExch(bd.overflow, 1);
            ok = tc_sync_and(done);
            // dW_l += dH_l^T A_l (M = 64 rows of DA, N = width of A_l, K = 128 samples)
            if (tid == 0 && ok) {
                if (l > 0)
                    mma_gemm<kTcTile>(tmem + dw_col<W, IN>(l), mnmajor(DA, kDaCols), mnmajor(HA + (l - 1) * L::ha, W),
                                      id_dw, !first_dw, kdw);
                else
                    mma_gemm<kTcTile>(tmem + dw_col<W, IN>(0), mnmajor(DA, kDaCols), mnmajor(XA, INP), id_dw0,
                                      !first_dw, kdw);
            }
        }
        if (!ok)
            break;
        // dX = dH_0 W_0 -> TMEM R0 (N = INP), then the hash scatter
        if (tid == 0) {
            mma_gemm<W>(tmem, kmajor(DA, kDaCols), mnmajor(Wt0, INP), id_dx, false);
            mma_commit(mbar);
        }
        const bool done_dx = mbar_poll(mbar, parity, bd.status);
        parity ^= 1u;
        first_dw = false;
        {
            const int s = srow;
            float g[16];
            if constexpr (INP / 2 == 16) {
                tmem_ld16(lane_base + half * 16, g);
            } else {
                float g8[8];
                tmem_ld8(lane_base + half * (INP / 2), g8);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    g[j] = g8[j];
            }
            const bool active = s < ns && done_dx;  // the whole warp scatters together
            if (split) {  // dL/d(encoding) to the scatter kernel, unscaled FP32, level-major
                if (active) {
                    float2 *dst = bd.sp_dx + (size_t)tile * kSplitDx;
                    const int l0 = half * (INP / 4);
#pragma unroll
                    for (int j = 0; j < INP / 4; ++j)
                        if (l0 + j < NL)
                            __stcs(dst + (l0 + j) * kTcTile + s,
                                   make_float2(g[2 * j] * inv_scale, g[2 * j + 1] * inv_scale));
                }
                ok = tc_sync_and(done_dx);
                continue;
            }
            float ph[3] = {0.f, 0.f, 0.f}, pl[3] = {0.f, 0.f, 0.f};
            if (active) {
                const float *rf = rayf + (s / nr) * kRayStride;
                const float t = ts[s];
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    pos_two_float(rf[RF_O + a], t, rf[RF_D + a], ph[a], pl[a]);
            }
            float2 *gtab = reinterpret_cast<float2 *>(od.grad);
            const int l0 = half * (INP / 4);
#pragma unroll
            for (int j = 0; j < INP / 4; ++j) {
                const int l = l0 + j;
                if (l >= NL)
                    break;
                const LevelDesc lv = od.lv[l];
                Corners cs;
                level_corners(lv, od.tmask, ph, pl, cs);
                PRENOM_CHECK_CORNERS(lv, od.tmask, cs, bd.status);
                scatter_level_warp(gtab + lv.offset, active, cs, g[2 * j] * inv_scale, g[2 * j + 1] * inv_scale,
                                   lane);
            }
        }
        ok = tc_sync_and(done_dx);
    }

    if (k >= 0 && ok)
        tc_flush_object<W, IN>(cur.od, cur.bd, lane_base, !first_dw, tc_dwo, dwo_acc, loss_acc, inv_scale, inv_enc);
    tc_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

template <int W, int IN, bool BF16>
cudaError_t launch_tc_t(const WorkItem &one, const WorkList &wl, int grid, cudaStream_t st)
{
    const size_t smem = TcLayout<W, IN>::bytes(wl.items ? wl.hmax : one.od.H, wl.split != 0);
    auto kern = wl.split ? fused_tc_kernel<W, IN, BF16, true> : fused_tc_kernel<W, IN, BF16, false>;
    cudaError_t e = allow_max_dynamic_smem(kern);
    if (e != cudaSuccess)
        return e;
    kern<<<grid, kThreads, smem, st>>>(one, wl);
    return cudaGetLastError();
}

// Resident CTAs per SM of a kernel variant for a launch whose deepest MLP has
// H hidden layers: as many as the SM's shared memory (each CTA's dynamic and
// static shared memory with the per-block reservation), its registers and its
// 512 TMEM columns hold (at least one, at most four).  A CTA holds its TMEM
// columns for its whole life, so a count the columns did not bound would leave
// the surplus CTAs waiting in their allocation.  0 when a device query fails.
template <int W, int IN, bool BF16>
int tc_occupancy_t(int H, bool split)
{
    cudaFuncAttributes fa{};
    int dev = 0, smem_sm = 0, reserved = 0, regs_sm = 0;
    auto kern = split ? fused_tc_kernel<W, IN, BF16, true> : fused_tc_kernel<W, IN, BF16, false>;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess)
        return 0;
    const size_t per_cta = TcLayout<W, IN>::bytes(H, split) + fa.sharedSizeBytes + (size_t)reserved;
    const long long regs_cta = (long long)((fa.numRegs + 7) / 8 * 8) * kThreads;
    const long long by_smem = (long long)smem_sm / (long long)per_cta, by_regs = regs_sm / regs_cta;
    const long long by_tmem = 512 / tc_cols<W, IN>(H, split);
    return (int)std::max(1LL, std::min(std::min(by_smem, by_regs), std::min(by_tmem, 4LL)));
}

template <bool BF16>
int tc_occupancy_prec(int W, int IN, int H, bool split)
{
#define PRENOM_TC_OCC(Wv, INv)                                                                                        \
    if (W == Wv && IN == INv)                                                                                         \
        return tc_occupancy_t<Wv, INv, BF16>(H, split);
    PRENOM_TC_OCC(16, 8)
    PRENOM_TC_OCC(16, 16)
    PRENOM_TC_OCC(16, 32)
    PRENOM_TC_OCC(32, 8)
    PRENOM_TC_OCC(32, 16)
    PRENOM_TC_OCC(32, 32)
    PRENOM_TC_OCC(64, 8)
    PRENOM_TC_OCC(64, 16)
    PRENOM_TC_OCC(64, 32)
#undef PRENOM_TC_OCC
    return 0;
}

template <bool BF16>
cudaError_t launch_tc_prec(const WorkItem &one, const WorkList &wl, int W, int IN, int grid, cudaStream_t st)
{
#define PRENOM_TC_CASE(Wv, INv)                                                                                       \
    if (W == Wv && IN == INv)                                                                                         \
        return launch_tc_t<Wv, INv, BF16>(one, wl, grid, st);
    PRENOM_TC_CASE(16, 8)
    PRENOM_TC_CASE(16, 16)
    PRENOM_TC_CASE(16, 32)
    PRENOM_TC_CASE(32, 8)
    PRENOM_TC_CASE(32, 16)
    PRENOM_TC_CASE(32, 32)
    PRENOM_TC_CASE(64, 8)
    PRENOM_TC_CASE(64, 16)
    PRENOM_TC_CASE(64, 32)
#undef PRENOM_TC_CASE
    return cudaErrorInvalidValue;
}

}  // namespace prenom
