// Internal descriptors and launchers of the PRENOM CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "prenom.h"

namespace prenom {

constexpr int kMaxLevels = 16;
constexpr int kThreads = 256;   // threads per CTA of the fused kernels
constexpr int kMaxNc = 256;     // prior probes per ray
constexpr int kMinNr = 4;       // samples per ray, lower bound (caps rays per tile)
constexpr int kMaxNr = 128;
constexpr int kMaxAdamSegs = 128;
constexpr int kMaxHidden = 3;   // hidden layers of an MLP, at most

// Bits of a launch's device status word: a bounded wait gave up, or (in a
// PRENOM_DEBUG_BOUNDS build) an index left its array and its access was skipped.
constexpr int32_t kStatusWait = 1, kStatusBounds = 2;

// Hash-grid level: resolution N_l, first entry of the level (in F-feature entries), dense flag.
struct LevelDesc {
    int32_t res;
    uint32_t offset;
    int32_t dense;
};

// One object's field as the fused kernel sees it.
struct ObjDesc {
    const float *theta;  // parameters (hash tables then MLP matrices)
    const uint32_t *feat16;  // BF16 copy of the hash tables (one bf16x2 word per entry), or NULL: gathers read theta
    float *grad;         // gradient accumulator (atomically added)
    int32_t L, IN, W, H;
    uint32_t tmask;      // T - 1 for hashed levels
    uint32_t mlp_off;    // float offset of W_1 in theta / grad
    LevelDesc lv[kMaxLevels];
    const float *grid;   // prior density grid [R][R][R], x fastest
    int32_t R;
    float lambda_d, lambda_sigma;
};

enum Mode : int32_t { kTrain = 0, kRender = 1, kRenderBwd = 2 };

// One batch of rays and what to do with it.
struct BatchDesc {
    int32_t n_rays, nc, nr, rays_per_tile, n_tiles;
    int32_t mode;
    float escape_eps, inv_r;
    const float *o, *d, *rgb, *depth;
    const uint8_t *is_obj;
    const float *c_rand, *u, *t_in;
    const float *upstream;  // [n][5] for kRenderBwd
    float *loss;            // device scalar, accumulated (kTrain)
    float *out_rgb, *out_depth, *out_acc, *out_t;
    float *out_sigma;       // optional [n][nr] density of every sample (render modes)
    int32_t *out_bins;
    uint64_t seed;
    uint32_t step, obj_id;
    // mixed-precision form only
    const float *loss_scale;  // device scalar multiplying dL/d(MLP output) before the 16-bit cast
    int32_t *overflow;        // device flag set when a scaled 16-bit gradient is not finite
    const float *enc_scale;   // FP16: device power of two multiplying the encoding before its 16-bit cast
                              // (divided out of the first layer's products in FP32); NULL = 1
    int32_t *status;          // device word: kStatusWait / kStatusBounds bits (below), zero when all is well
    // split execution of a mixed-precision training step (all NULL otherwise):
    // the three kernels hand over these per-batch buffers
    float *sp_t;    // [n_rays][nr] sample depths
    float *sp_rays; // [n_tiles][kTcRayMax][16] each ray's data as the tensor-core kernel keeps it
    uint4 *sp_x;    // [n_tiles][kSplitXBytes / 16] each tile's encoding: 16-bit in the MMA operand
                    // layout (tensor-core kernel) or FP32 feature-major [IN][kSplitTile] (FP32 kernel)
    float2 *sp_dx;  // [n_tiles][kMaxLevels][kSplitTile] dL/d(encoding), FP32, level-major
};

constexpr int kSplitTile = 128;                      // samples per tile of the mixed-precision kernels
constexpr int kSplitXBytes = kSplitTile * 32 * 4;    // encoding image of a tile (width <= 32, up to FP32)
constexpr int kSplitDx = kMaxLevels * kSplitTile;    // float2 per tile of dL/d(encoding)
constexpr int kTcRayMax = kSplitTile / kMinNr;       // rays per tile at most
constexpr int kSplitRayFloats = kTcRayMax * 16;      // floats per tile of ray data

// Dynamic loss-scaling state of one mixed-precision object (device memory).
struct LossScaleState {
    float scale;
    int32_t good_steps;
    int32_t overflow;
    int32_t skipped;
    int32_t growth_interval;  // clean steps in a row after which the scale doubles
    // FP16 objects: the encoding and with it every hidden activation (the layers
    // have no biases, ReLU is positively homogeneous) are cast to FP16 scaled by
    // enc_scale = 2^k, k = floor(log2(kEncTarget / (A G))) in [kEncMinLog2,
    // kEncMaxLog2], A = max |hash entry| (the encoding is a convex combination of
    // entries, so |e| <= A) and G = max(1, max_l prod_{j<=l} ||W_j||_inf) over the
    // hidden layers (|h_l| <= |h_{l-1}|_max ||W_l||_inf): no scaled value exceeds
    // kEncTarget, and the small values of a fresh object stay FP16 normals
    int32_t enc_auto;      // 1 for FP16 objects (else enc_scale stays 1)
    float enc_scale;
    uint32_t hash_absmax;  // bits of max |hash entry| gathered by the last pass over theta
    const float *mlp;      // the object's MLP matrices in theta (W_1 [W][IN], W_2..W_H [W][W])
    int32_t in, width, hidden;
};
constexpr int32_t kLossScaleGrowth = 1000;  // default growth interval
constexpr float kEncTarget = 32768.f;       // bound on every scaled value, half of FP16's 65504
constexpr int kEncMinLog2 = -16, kEncMaxLog2 = 24;

struct WorkItem;
struct WorkList;

// Mixed-precision fused kernel (tcgen05 MLP); precision 1 = FP16, 2 = BF16.
size_t fused_tc_smem(int W, int IN, int H, bool split);
// Resident CTAs per SM (1 or 2; 0 if the variant does not fit) of the tensor-core kernel.
int fused_tc_occupancy(int precision, int W, int IN, int H, bool split);
cudaError_t launch_fused_tc(const ObjDesc &od, const BatchDesc &bd, int precision, int grid, cudaStream_t st);
cudaError_t launch_fused_tc_list(const WorkList &wl, int W, int IN, int precision, int grid, cudaStream_t st);
cudaError_t launch_fused_tc_bf16(const WorkItem &one, const WorkList &wl, int W, int IN, int grid, cudaStream_t st);
cudaError_t launch_fused_tc_fp16(const WorkItem &one, const WorkList &wl, int W, int IN, int grid, cudaStream_t st);
// Split execution of a mixed-precision training step: sampling + encoding,
// then the tensor-core kernel without its scatter, then the hash scatter.
// wl.items == nullptr means the single item `one`.
// per_sm: 4 or 3 resident CTAs per SM (the registers budget of the variant; the
// grid is sized by the caller to match)
cudaError_t launch_sample_encode(const WorkItem &one, const WorkList &wl, int precision, int per_sm, int grid,
                                 cudaStream_t st);
// whole_runs: lanes of one cell summed over whole runs instead of chunks of four.
cudaError_t launch_hash_scatter(const WorkItem &one, const WorkList &wl, int grid, cudaStream_t st,
                                bool whole_runs = false);
// Bytes of split buffers for a batch of n_rays rays of nr samples in n_tiles tiles.
inline size_t split_bytes(int n_rays, int nr, int n_tiles)
{
    const size_t t = ((size_t)n_rays * nr * sizeof(float) + 255) / 256 * 256;
    return t + (size_t)n_tiles * (kSplitXBytes + kSplitDx * 8 + kSplitRayFloats * 4);
}
// Loss-scale bookkeeping after the Adam step of a mixed-precision object.
cudaError_t launch_loss_scale_update(LossScaleState *s, cudaStream_t st);
constexpr int kMaxScaleObjs = 256;
struct ScaleList {
    int32_t n;
    LossScaleState *s[kMaxScaleObjs];
};
cudaError_t launch_loss_scale_update_list(const ScaleList &l, cudaStream_t st);
// mirror[i] = bf16(theta[i]) for i < n (after any write of theta other than Adam's).
cudaError_t launch_mirror_refresh(const float *theta, int64_t n, uint16_t *mirror, int grid, cudaStream_t st);
// enc_scale of an FP16 object from max |theta[0..n_hash)| (after any write of
// theta other than Adam's, which gathers the maximum as it updates).
cudaError_t launch_enc_scale_refresh(const float *theta, int64_t n_hash, LossScaleState *s, int grid,
                                     cudaStream_t st);
// Zeroes the loss accumulator of every item of a device work list.
cudaError_t launch_zero_losses(const WorkItem *items, int n, cudaStream_t st);

// One unit of work of a fused launch: an object's field, one batch of its
// rays, and the launch-wide index of the batch's first tile.
struct WorkItem {
    ObjDesc od;
    BatchDesc bd;
    int32_t tile_begin;
};

// The work of a batched launch (all items share the MLP width and encoding
// width; hidden depths may differ, hmax is the deepest).  items == nullptr
// means a single item passed by value.
struct WorkList {
    const WorkItem *items;  // device memory
    int32_t n_items, total_tiles, hmax;
    int32_t split;  // 1: sampling, encoding and the hash scatter run in kernels of their own
    int32_t feat16; // 1: every item's gathers read the BF16 copy of its tables (ObjDesc::feat16)
};

// Dynamic shared memory (bytes) of the fused FP32 kernel for (W, IN, H, S).
size_t fused_fp32_smem(int W, int IN, int H, int S);
// Largest tile (128 or 64 samples) whose shared memory fits; 0 if none.
int fused_fp32_pick_tile(int W, int IN, int H, size_t smem_limit);
// Launches the fused kernel on one object; returns the CUDA error of the launch.
cudaError_t launch_fused_fp32(const ObjDesc &od, const BatchDesc &bd, int S, int grid, cudaStream_t st);
// Launches the fused kernel on a work list of objects of one (W, IN).
cudaError_t launch_fused_fp32_list(const WorkList &wl, int W, int IN, int S, int grid, cudaStream_t st);
cudaError_t launch_fused_fp32_w16(const WorkItem &one, const WorkList &wl, int IN, int S, int grid, cudaStream_t st);
cudaError_t launch_fused_fp32_w32(const WorkItem &one, const WorkList &wl, int IN, int S, int grid, cudaStream_t st);
cudaError_t launch_fused_fp32_w64(const WorkItem &one, const WorkList &wl, int IN, int S, int grid, cudaStream_t st);

// Adam over up to kMaxAdamSegs parameter spans.
struct AdamSeg {
    float *theta, *grad, *m, *v;
    int64_t n;
    float lr_c1;     // lr / (1 - beta1^t)
    float inv_c2;    // 1 / (1 - beta2^t)
    const int32_t *skip;  // mixed precision: nonzero overflow flag = drop this step (NULL for FP32)
    const float2 *scal;   // device (lr_c1, inv_c2) of this step, or NULL to use the two fields above
    uint32_t *absmax;     // FP16: max |updated theta| over [0, n_hash) gathered here (NULL = not gathered)
    int64_t n_hash;
    uint16_t *mirror;     // BF16 copy of theta[0, n_hash) written with the update (NULL = none)
};
struct AdamArgs {
    int32_t n_segs;
    float beta1, beta2, eps;
    int64_t chunk_start[kMaxAdamSegs + 1];  // prefix sums of per-segment chunk counts
    AdamSeg seg[kMaxAdamSegs];
};
constexpr int kAdamChunk = 1024;  // floats per chunk (fine enough that the last wave leaves no long tail)
cudaError_t launch_adam(const AdamArgs &a, int grid, cudaStream_t st);

// Reptile meta step (§III-A): broadcast of the meta-parameters to the task
// objects (with zeroed gradient and Adam state), the task sum, and the outer
// update of Eq. 2.
constexpr int kMaxReptileTasks = 128;
enum ReptileOp : int { kReptileBroadcast = 0, kReptileSum = 1, kReptileApply = 2 };
struct ReptileArgs {
    int32_t n_tasks;
    int64_t n;       // parameters
    int64_t n_pad;   // stride of the arrays in a task's arena (a multiple of 64)
    float beta, nf;  // step size and the total number of tasks (as float)
    float *meta;     // meta theta (broadcast source; updated by sum-with-meta and apply)
    float *sum;      // task sum (output of a sum without meta, input of apply)
    float *theta[kMaxReptileTasks];  // each task's arena: theta, grad, m, v at n_pad strides
};
cudaError_t launch_reptile(const ReptileArgs &a, int op, int grid, cudaStream_t st);

// Training rays from keyframes: candidate count, scan, compaction and the draws.
size_t make_rays_scratch(int64_t n_pix);
cudaError_t launch_make_rays(const prenom_keyframe *d_kf, const int64_t *d_pix_off, int n_kf, int64_t n_pix,
                             const prenom_object_state &st, unsigned char *scratch, int n_rays, const uint32_t *draws,
                             uint64_t seed, uint32_t call, float *o, float *d, float *rgb, float *depth,
                             uint8_t *is_obj, int64_t **d_count, cudaStream_t st_);

// Prior density grid support: query rays of an R^3 grid of voxel centres, and
// the yaw scores of Eq. 3 (one block per yaw sample, FP64 sums).
cudaError_t launch_density_rays(int R, float *o, float *d, float *t, cudaStream_t st);
cudaError_t launch_yaw_scores(const float *grid, int R, const float *P, int n, int n_gamma, double *score,
                              cudaStream_t st);

// Random initialisation of theta: hash entries U(-1e-4, 1e-4), MLP Xavier-uniform.
cudaError_t launch_init_params(float *theta, int64_t n_hash, const int32_t *mlp_shape /*[2*(H+1)]*/,
                               int n_layers, uint64_t seed, uint32_t obj, int grid, cudaStream_t st);

}  // namespace prenom
