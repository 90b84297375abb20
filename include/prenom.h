/* prenom.h — C ABI of the GB300 (sm_103a) object-NeRF training library.
 *
 * The library implements the hot path of the online object mapper of
 * "Category-level Meta-learned NeRF Priors for Efficient Object Mapping"
 * (PRENOM, arXiv 2503.01582): one training step of many small object-level
 * NeRFs (§III-B), made of
 *   (a) probabilistic ray sampling over a prior density grid
 *       (§III-B "Probabilistic Ray Sampling", Eq. 4-6, escape rule),
 *   (b) a multiresolution hash-grid encoding and a shallow MLP
 *       (§III-B "Object-level NeRFs"),
 *   (c) volume rendering and the RGB-D loss (§III-B "Volume Rendering",
 *       Eq. 7-9),
 *   (d) the backward pass and an Adam update (last sentence of §III-B).
 *
 * Conventions for every call:
 *   - return 0 (PRENOM_OK) on success or a negative PRENOM_ERR_* code; the
 *     message of the last failure is available from prenom_last_error();
 *     no C++ exception crosses this interface;
 *   - all work is stream-ordered on the stream given to prenom_create();
 *     calls return before the GPU has finished unless stated otherwise;
 *   - pointers marked "device" must be CUDA device (or managed) memory that
 *     stays valid until the stream reaches the call's work; the library
 *     never frees or keeps them;
 *   - the library owns every object's parameters theta, gradients and Adam
 *     moments, allocated once by prenom_create_object();
 *   - one context belongs to one host thread at a time (no internal locks).
 *
 * Parameter vector layout of one object (what prenom_get_state copies):
 * hash tables level by level, each level entry-major with F features per
 * entry and padded to a multiple of 8 entries (prenom_level_info gives the
 * offsets; padding entries are never read and never change), then one
 * row-major (out x in) matrix per MLP layer: W_1 [W][L*F], W_2 .. W_H [W][W],
 * W_out [4][W]; no biases.
 */
#ifndef PRENOM_H
#define PRENOM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PRENOM_API __attribute__((visibility("default")))
#else
#define PRENOM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define PRENOM_OK 0
#define PRENOM_ERR_INVALID_ARG (-1)    /* bad pointer, size, index or architecture */
#define PRENOM_ERR_OOM (-2)            /* a device allocation failed */
#define PRENOM_ERR_CUDA (-3)           /* a CUDA runtime call or a launch failed */
#define PRENOM_ERR_DEVICE_TIMEOUT (-4) /* a bounded device-side wait gave up */
#define PRENOM_ERR_NONFINITE (-5)      /* a checked loss was NaN or infinite */
#define PRENOM_ERR_DEVICE_BOUNDS (-6)  /* debug build: an index left its array (access skipped) */

/* Debug build.  The same sources compiled with -DPRENOM_DEBUG_BOUNDS make
 * libprenom_debug.so (paper_2503_01582_gb300.build.build(debug_bounds=True)),
 * with the same entry points.  Its kernels test every hash-table corner index
 * against its level's entry count, every prior-grid voxel index against R^3
 * and every ray index against the batch's ray count where the index is
 * formed; an index outside skips its access and marks the context's device
 * status word, which prenom_sync() reports as PRENOM_ERR_DEVICE_BOUNDS.  No
 * check traps or faults.  The regular library has no such tests: its indices
 * are in range by construction (positions clamped to the unit cube, cells to
 * the level's resolution, hashes masked to T - 1, rays counted from the batch). */

#define PRENOM_PRECISION_FP32 0 /* FP32 features, MLP and accumulation */
/* Mixed precision: the MLP runs on the tensor cores with 16-bit operands and
 * FP32 accumulation; parameters, Adam state, hash features, sampling,
 * transmittance and the loss stay FP32.  FP16 uses a dynamic loss scale
 * (initial 2^15, halved and the step dropped on an overflow, doubled after 1000
 * clean steps, see prenom_set_loss_scale); BF16 uses a scale of 1. */
#define PRENOM_PRECISION_FP16 1
#define PRENOM_PRECISION_BF16 2

/* prenom_arch.features: what the hash-grid gathers of the encoding read.
 * FP32: the FP32 parameter tables themselves.  BF16 (mixed-precision objects
 * only): a BF16 copy of the tables that each Adam step writes beside the FP32
 * master values (and that every other write of theta refreshes); the gathers
 * read it, four entries to one 16-byte load where the x-adjacent corners share
 * it, and the encoding is summed in FP32.  Gradients, Adam and the master
 * values stay FP32 in both. */
#define PRENOM_FEATURES_FP32 0
#define PRENOM_FEATURES_BF16 2

/* prenom_train_opts.flags */
#define PRENOM_FLAG_NO_ADAM 1u      /* accumulate gradients, skip Adam (step count unchanged) */
#define PRENOM_FLAG_CHECK_FINITE 2u /* synchronise and fail with NONFINITE on a NaN/inf loss (per-object path) */
#define PRENOM_FLAG_NO_GRAPH 4u     /* batched steps: launch directly instead of replaying a captured graph */
#define PRENOM_FLAG_FUSED 8u        /* training: one fused kernel per step and group instead of the split
                                       form (sampling+encoding, the MLP kernel, hash scatter as three
                                       kernels); the results agree to rounding order */
#define PRENOM_FLAG_SPLIT 16u       /* training: always the split form (not tuned) */
#define PRENOM_FLAG_RETUNE 32u      /* prenom_autotune: forget the step's earlier tuning and tune it again
                                       (ignored by the training calls) */
#define PRENOM_FLAG_CONCURRENT 64u  /* batched steps of several groups on a non-default stream: run the
                                       groups concurrently on side streams, each followed by the Adam pass
                                       of its own objects, without the autotuner's trial of one after the
                                       other against concurrently; the results are the same either way */

/* prenom_get_state / prenom_set_state: which buffer */
#define PRENOM_STATE_THETA 0
#define PRENOM_STATE_GRAD 1
#define PRENOM_STATE_ADAM_M 2
#define PRENOM_STATE_ADAM_V 3

/* Kernel ids for the timing interface. */
#define PRENOM_KERNEL_TRAIN 0  /* fused sample+encode+MLP+render+loss+backward (split form: MLP+render+loss+MLP backward) */
#define PRENOM_KERNEL_ADAM 1   /* dense Adam over every parameter of the step's objects */
#define PRENOM_KERNEL_RENDER 2 /* forward only */
#define PRENOM_KERNEL_RENDER_BWD 3
#define PRENOM_KERNEL_INIT 4   /* random parameter initialisation */
#define PRENOM_KERNEL_SAMPLE_ENCODE 5 /* split form: prior sampling + hash encoding */
#define PRENOM_KERNEL_SCATTER 6       /* split form: hash-grid scatter of the encoding's gradient */
#define PRENOM_N_KERNELS 7

typedef struct prenom_ctx prenom_ctx; /* opaque; owns all device state */

/* Architecture alpha of one object NeRF (§III-A "Architecture Optimization"
 * lists hash-grid and MLP hyper-parameters and lambda_d, lambda_sigma).
 * Supported values: F = 2; L in {4, 8, 16}; width in {16, 32, 64};
 * 1 <= hidden <= 3; 8 <= log2T <= 24; 2 <= n_min <= n_max <= 2^20;
 * precision = PRENOM_PRECISION_FP32, _FP16 or _BF16; features =
 * PRENOM_FEATURES_FP32, or _BF16 with a mixed precision. */
typedef struct {
    int32_t L, F, log2T, n_min, n_max; /* levels, features/level, log2 table size, resolutions */
    int32_t width, hidden;             /* MLP hidden width W and hidden layer count H */
    int32_t precision;                 /* PRENOM_PRECISION_* */
    float lambda_d, lambda_sigma;      /* Eq. 9 loss weights */
    int32_t features;                  /* PRENOM_FEATURES_* (0 = FP32) */
} prenom_arch;

/* Step options.  lr, beta1, beta2, eps: Adam (§III-B).  nc, nr: probes and
 * samples per ray (§III-B, N_c and N_r; 4 <= nr <= 128, 1 <= nc <= 256).
 * escape_eps: the escape threshold epsilon of §III-B (the paper uses 1e-4).
 * loss_scale_init: for a mixed-precision object, when > 0, the loss scale it
 * starts from at its first step (0 = the default of its precision; ignored
 * in FP32).  flags: PRENOM_FLAG_*. */
typedef struct {
    float lr, beta1, beta2, eps;
    int32_t nc, nr;
    float escape_eps;
    float loss_scale_init;
    uint32_t flags;
} prenom_train_opts;

/* One object's rays for one step, in the object's normalized frame (the
 * unit cube of §III-A; rays "transformed into the object frame", §III-B).
 * All arrays are device memory, row-major, n_rays rows:
 *   o, d      [n][3] float  origin and direction (d need not be unit; t is in units of |d|)
 *   rgb       [n][3] float  target colour C(r) of object rays (read for R_o only)
 *   depth     [n]    float  target depth D(r) of object rays (read for R_o only)
 *   is_obj    [n]    uint8  1 = ray of R_o (hits the object), 0 = R_b (background)
 *   c_rand    [n][3] float  background supervision colour C_rand, or NULL to draw it
 *                           from the library's Philox stream (seed, step, obj, ray)
 *   uniforms  [n][nr] float stratified uniforms in [0,1) for the inverse transform,
 *                           sorted along each ray, or NULL to draw them from Philox
 *   t_in      [n][nr] float optional sample depths, sorted, inside the ray's box
 *                           interval; when non-NULL the prior sampler is skipped
 *                           (uniforms are then ignored). */
typedef struct {
    int32_t obj;
    int32_t n_rays;
    const float *o, *d;
    const float *rgb, *depth;
    const uint8_t *is_obj;
    const float *c_rand;
    const float *uniforms;
    const float *t_in;
} prenom_ray_batch;

/* Creates a context on the current CUDA device.  cuda_stream: a cudaStream_t
 * (NULL = the legacy default stream) on which all work is ordered; seed keys
 * the Philox stream used when a batch omits uniforms or c_rand and for random
 * initialisation.  *out receives the context (NULL on failure). */
PRENOM_API int prenom_create(prenom_ctx **out, void *cuda_stream, uint64_t seed);

/* Destroys a context, its objects and device buffers (synchronises first). */
PRENOM_API void prenom_destroy(prenom_ctx *ctx);

/* The message of the last failing call on ctx ("" if none; ctx may be NULL,
 * then the message of the last failed prenom_create is returned). */
PRENOM_API const char *prenom_last_error(const prenom_ctx *ctx);

/* Registers one object NeRF (§III-B "Object-level NeRFs": a known category
 * loads its meta-learned theta, an unknown one uses random initialisation).
 * init_params: host or device pointer to param_count floats in the layout
 * above (copied), or NULL for random initialisation (hash entries uniform in
 * [-1e-4, 1e-4], MLP matrices Xavier-uniform, from the context's Philox
 * stream).  Gradients and Adam moments start at zero, the step count at 0.
 * Allocates the object's device arena (4 x param_count floats). */
PRENOM_API int prenom_create_object(prenom_ctx *ctx, const prenom_arch *arch, const float *init_params,
                         int32_t *obj_out);

/* Frees an object's device memory; its id is not reused. */
PRENOM_API int prenom_destroy_object(prenom_ctx *ctx, int32_t obj);

/* Number of floats in the object's parameter vector. */
PRENOM_API int prenom_param_count(prenom_ctx *ctx, int32_t obj, size_t *n);

/* Number of floats in the parameter vector of architecture arch (host
 * pointer; the same rules as prenom_create_object, PRENOM_ERR_INVALID_ARG
 * otherwise), without a context or any device work: for sizing caller-owned
 * state (prenom_train_step_noalloc) and balancing objects across GPUs. */
PRENOM_API int prenom_arch_param_count(const prenom_arch *arch, size_t *n);

/* Level geometry of the hash grid, for checking the layout contract:
 * res[l] = N_l, offset[l] = float offset of level l in theta (l = 0..L;
 * offset[L] = offset of W_1), dense[l] = 1 if level l is stored densely. */
PRENOM_API int prenom_level_info(prenom_ctx *ctx, int32_t obj, int32_t *res, int64_t *offset, int32_t *dense);

/* Sets the prior density grid F (§III-A "Normalized mesh generation", used by
 * §III-B sampling): res^3 floats, x fastest, value of the voxel centred at
 * ((i+1/2)/res, (j+1/2)/res, (k+1/2)/res); finite and >= 0; res >= 2.
 * grid: host or device pointer, copied (the caller keeps ownership). */
PRENOM_API int prenom_set_prior_grid(prenom_ctx *ctx, int32_t obj, const float *grid, int32_t res);

/* One training step (§III-B): for every batch, sample, encode, run the MLP,
 * composite, form the loss of Eq. 9 averaged over that batch's rays, and
 * back-propagate into the object's gradient buffer; then one Adam step for
 * every distinct object named by the batches (unless PRENOM_FLAG_NO_ADAM).
 * Gradients are zeroed by the Adam step, so NO_ADAM steps accumulate.
 * Several batches form the batched form (§IV-A trains objects in parallel):
 * the batches are grouped by kernel variant (precision, width, encoding
 * width) and each group runs as ONE persistent launch over a work list
 * spanning all its objects (or, in the split form, sampling + encoding, the
 * MLP kernel and the hash scatter as three launches over the same list); one
 * Adam launch then updates every object (when the step's groups run
 * concurrently, one Adam launch per group, on the group's stream after its
 * kernels).
 * A single batch takes the same path.  The first calls of a new group
 * signature (kernel variant, and batch and tile counts rounded down to powers
 * of two; one untimed call, then three rounds over the candidates, each
 * candidate judged by its median) try the
 * split form and several work-chunk sizes (tiles per CTA) and keep the
 * fastest; a step of several groups on a non-default stream then times its
 * groups one after the other and concurrently on side streams (three rounds
 * each) and keeps the faster; afterwards, on a non-default stream and with timing off, the whole
 * step is captured once per exact signature as a CUDA graph and replayed
 * (PRENOM_FLAG_NO_GRAPH disables the graph); a context keeps at most 64
 * graphs, evicting the least recently used after waiting for its stream.
 * A step synchronises with the step before the previous
 * one (two staging buffers are in flight), allocates its work-list and split
 * buffers on first use and when they must grow, and updates at most 128
 * objects.  The tuning calls and the first capture of a signature can be
 * taken out of a training loop by calling prenom_autotune() first.
 * With PRENOM_FLAG_CHECK_FINITE the batches run one launch each, without
 * tuning or graphs; the call then waits for the stream and, when a batch's
 * loss is NaN or infinite, clears the gradients of the step's objects, takes
 * no Adam step and returns PRENOM_ERR_NONFINITE (with loss_dev NULL at most
 * 64 batches, whose losses go to the context's own scratch).
 * loss_dev: device [n_batches] floats receiving each batch's loss, or NULL.
 * Each object named must have a prior grid unless every batch naming it
 * gives t_in. */
PRENOM_API int prenom_train_step(prenom_ctx *ctx, const prenom_ray_batch *batches, int32_t n_batches,
                      const prenom_train_opts *opts, float *loss_dev);

/* Forward rendering of one batch (§III-B "Volume Rendering", Eq. 7): colour
 * rgb [n][3], depth [n], accumulated opacity acc [n] (sum of the weights), all
 * device, any may be NULL.  bins_out [n][nr] int32 (0-based prior bin of each
 * sample, -1 when t_in was given) and t_out [n][nr] (sample depths) are
 * optional. */
PRENOM_API int prenom_render(prenom_ctx *ctx, const prenom_ray_batch *batch, const prenom_train_opts *opts,
                  float *rgb, float *depth, float *acc, int32_t *bins_out, float *t_out);

/* Adjoint of prenom_render for upstream gradients d_out [n][5] (dL/dC[3],
 * dL/dD, dL/dA per ray, device): adds dL/dtheta into grad (device,
 * param_count floats, caller-owned, accumulated, not zeroed, 16-byte aligned
 * or PRENOM_ERR_INVALID_ARG). */
PRENOM_API int prenom_render_backward(prenom_ctx *ctx, const prenom_ray_batch *batch,
                           const prenom_train_opts *opts, const float *d_out, float *grad);

/* Blocking copies of one object buffer (which = PRENOM_STATE_*) to / from
 * host or device memory; n must equal param_count. */
PRENOM_API int prenom_get_state(prenom_ctx *ctx, int32_t obj, int32_t which, float *dst, size_t n);
PRENOM_API int prenom_set_state(prenom_ctx *ctx, int32_t obj, int32_t which, const float *src, size_t n);

/* Adam step count of an object (bias correction uses step + 1 next). */
PRENOM_API int prenom_get_step(prenom_ctx *ctx, int32_t obj, int32_t *step);
PRENOM_API int prenom_set_step(prenom_ctx *ctx, int32_t obj, int32_t step);

/* ------------------------------------------------- meta-learning (§III-A)
 * One Reptile meta step over a meta-batch of tasks (§III-A "Meta-learning"):
 * every task object starts from the meta object's parameters with fresh Adam
 * state, takes q inner training steps on its own reconstruction task (Eq. 1;
 * the inner optimiser is the Adam step of prenom_train_step, whose batched
 * form trains all tasks of the meta-batch in one launch per step), and the
 * meta-parameters then move toward the tasks' result:
 *     theta <- theta + beta (mean_t theta_t^(q) - theta)
 * (the batched reading of Eq. 2; with one task it is Eq. 2 itself).  Meta and
 * task objects are ordinary objects of one architecture (L, F, T, N_min,
 * N_max, width, depth; their precisions may differ); at most 128 tasks, each
 * listed once, the meta object not among them.  Stream-ordered, no
 * synchronisation.  Errors: PRENOM_ERR_INVALID_ARG for a bad object list or
 * beta outside [0, 1].
 *
 * prenom_reptile_begin: theta_t <- theta_meta, gradient and Adam moments of
 *   every task zeroed, its step count reset to 0 (its loss scale is kept).
 * prenom_reptile_update: the outer update above over the n_tasks tasks (their
 *   sum in task order, FP32), in one pass.
 * Across several GPUs the tasks are split between ranks: each rank calls
 * prenom_reptile_task_sum (sum: device, param_count floats, 16-byte aligned,
 * overwritten with the sum of its tasks' parameters), the ranks add their sums
 * (one all-reduce), and each calls prenom_reptile_apply with n_total = the
 * number of tasks over all ranks. */
PRENOM_API int prenom_reptile_begin(prenom_ctx *ctx, int32_t meta, const int32_t *tasks, int32_t n_tasks);
PRENOM_API int prenom_reptile_update(prenom_ctx *ctx, int32_t meta, const int32_t *tasks, int32_t n_tasks,
                                     float beta);
PRENOM_API int prenom_reptile_task_sum(prenom_ctx *ctx, const int32_t *tasks, int32_t n_tasks, float *sum);
PRENOM_API int prenom_reptile_apply(prenom_ctx *ctx, int32_t meta, const float *sum, int32_t n_total, float beta);

/* ------------------------------------------------ training rays (§III-B)
 * §III-B "Training Data": RGB-D images, instance masks and camera poses of the
 * keyframes supervise the object; "Probabilistic Ray Sampling": camera rays
 * are transformed into the object frame with the estimated object pose and
 * bounded by the object's box.  prenom_make_rays turns keyframes into a ray
 * batch of prenom_ray_batch's layout:
 *   - object frame: p_n = R_wo^T (p_w - centre) / size + 1/2 (the normalised
 *     frame of Eq. 3: the box is the unit cube); the world ray parameter t is
 *     kept, so o = R_wo^T (t_wc - centre) / size + 1/2 and d = R_wo^T d_w / size
 *     with d_w the unit world direction of the pixel;
 *   - pixel (x, y) shoots through (x + 1/2, y + 1/2) of a pinhole camera:
 *     camera direction ((x+1/2-cx)/fx, (y+1/2-cy)/fy, 1), rotated by R_wc;
 *   - a pixel is a candidate when its ray meets the box and, when its mask
 *     equals state->instance (an object ray, is_obj = 1), its depth is > 0 and
 *     finite; other candidates are background rays (is_obj = 0);
 *   - rgb target = rgb / 255; depth target of an object ray = z-depth times
 *     |(x', y', 1)| (the distance t along the ray), 0 for background rays;
 *   - n_rays rays are drawn uniformly from all candidates of all keyframes
 *     (keyframe-major, row-major order): ray j takes candidate
 *     floor(r_j n_candidates / 2^32), r_j = draws[j] (device uint32) or, with
 *     draws NULL, word j mod 4 of Philox4x32-10(ctr = (j / 4, 0, call,
 *     0x52415953), key = the context seed), call counting this context's
 *     prenom_make_rays calls from 0;
 *   - with no candidate every ray is o = (-1, -1, -1), d = 0, which misses
 *     the box and renders to zero.
 * The geometry is FP32 with every operation rounded (no contraction), in the
 * order the formulas above are written.  keyframes and state: host; image
 * pointers inside: device (rgb [height][width][3] u8, depth [height][width]
 * FP32 z-depth, mask [height][width] int32).  o, d, rgb: device [n_rays][3];
 * depth: device [n_rays]; is_obj: device [n_rays] u8 (all caller-owned).
 * n_candidates: host, receives the candidate count when non-NULL (the call
 * then waits for the stream).  At most 4096 keyframes and 2^31 - 1 pixels. */
typedef struct {
    int32_t width, height;
    const uint8_t *rgb;
    const float *depth;
    const int32_t *mask;
    float fx, fy, cx, cy; /* pinhole intrinsics in pixels */
    float R_wc[9];        /* camera-to-world rotation, row-major (columns: camera x, y, viewing axis) */
    float t_wc[3];        /* camera centre in the world */
} prenom_keyframe;

typedef struct {
    int32_t instance;     /* mask id of the object */
    float R_wo[9];        /* object-to-world rotation, row-major */
    float centre[3];      /* world position of the box centre */
    float size[3];        /* box extents along the object axes (> 0) */
} prenom_object_state;

PRENOM_API int prenom_make_rays(prenom_ctx *ctx, const prenom_keyframe *keyframes, int32_t n_keyframes,
                                const prenom_object_state *state, int32_t n_rays, const uint32_t *draws, float *o,
                                float *d, float *rgb, float *depth, uint8_t *is_obj, int64_t *n_candidates);

/* ------------------------------------------- prior density grid (§III-A, §III-B)
 * prenom_density_grid: the object's density field sampled at the centres of
 * an res^3 grid over the unit cube (§III-A "Normalized mesh generation": the
 * NeRF's density output over a cubic grid of resolution R is the prior density
 * grid): grid_out[(k res + j) res + i] = exp(min(o_0, 15)) at
 * ((i+1/2)/res, (j+1/2)/res, (k+1/2)/res), x fastest -- the layout
 * prenom_set_prior_grid takes.  grid_out: device, res^3 floats, caller-owned;
 * 4 <= res <= 64.  Computed by the object's own forward kernel (a mixed-
 * precision object evaluates its MLP in its 16-bit format).  Stream-ordered.
 * prenom_refresh_prior: the same density written over the object's prior
 * grid (§III-B updates the prior every m iterations so that sampling follows
 * the object as it is learnt); the grid is reallocated if res changes.
 *
 * prenom_canonical_yaw: Eq. 3 (§III-B "Object State Canonicalization") with
 * the object's prior grid: for gamma_g = 2 pi g / n_gamma, g < n_gamma, the
 * cloud points (device, [n_points][3] FP32, object frame centred on the
 * object, z up) is turned about z by gamma_g, centred at the midpoint of its
 * extents and divided by them (+1/2, an axis of zero extent maps to 1/2), and
 * scored by the sum of the prior's trilinear density over its points (each
 * lookup FP32, the sum FP64 in a fixed order).  best (host) receives the first
 * g of largest score; scores (host or device, n_gamma floats) may be NULL.
 * Blocking (reads the scores back).  n_gamma <= 65536. */
PRENOM_API int prenom_density_grid(prenom_ctx *ctx, int32_t obj, int32_t res, float *grid_out);
PRENOM_API int prenom_refresh_prior(prenom_ctx *ctx, int32_t obj, int32_t res);
PRENOM_API int prenom_canonical_yaw(prenom_ctx *ctx, int32_t obj, const float *points, int32_t n_points,
                                    int32_t n_gamma, float *scores, int32_t *best);

/* Runs, ahead of training, what the first calls of prenom_train_step() with
 * these batches and options would otherwise do inside the training loop: the
 * autotuner's calls for every group signature not yet tuned (one untimed call,
 * then three rounds over the candidates) and for the step-level choice between
 * its groups one after the other and forked, run as gradient-only steps -- no Adam
 * update, no change of theta, Adam moments or step counts; the gradients they
 * accumulate and any 16-bit overflow flag they raise are cleared afterwards --
 * and the capture of the step's CUDA graph for both staging buffers (when
 * graphs apply: a non-default stream, timing off, no PRENOM_FLAG_NO_GRAPH).
 * The next prenom_train_step() calls with batches of the same signature then
 * replay without tuning or capturing.  Same arguments and checks as
 * prenom_train_step(); batches with PRENOM_FLAG_CHECK_FINITE are neither tuned
 * nor captured, so the call does nothing for them.  With PRENOM_FLAG_RETUNE
 * the step's groups and its step-level choice are tuned again (the relative
 * costs of the candidates move as objects train: once surfaces turn opaque
 * the samples behind them carry no gradient and the scatter has less to do),
 * and graphs are
 * captured for the new choices.  Waits for the stream. */
PRENOM_API int prenom_autotune(prenom_ctx *ctx, const prenom_ray_batch *batches, int32_t n_batches,
                               const prenom_train_opts *opts);

/* Counters of the context: step graphs captured so far, and training steps run
 * as autotuner measurements (either may be NULL).  Unchanged counters around a
 * loop of steps show that the loop neither tuned nor captured. */
PRENOM_API int prenom_capture_count(prenom_ctx *ctx, int64_t *captures, int64_t *tuning_calls);

/* Per-group kernel times of the batched steps run while timing was enabled
 * (prenom_enable_timing): one line per (group, kernel) "label<TAB>kK<TAB>total
 * ms<TAB>launches", where the label names the group's precision, MLP width W,
 * encoding width IN, deepest hidden depth H, batch and tile counts, form
 * (split or fused) and grid, and K is a PRENOM_KERNEL_* id.  Synchronises.
 * buf: host, cap bytes, NUL-terminated, truncated to fit. */
PRENOM_API int prenom_timing_report(prenom_ctx *ctx, char *buf, size_t cap);

/* The autotuner's record as text (one line per group signature: the group's
 * own device time in ms (its launches, between events) in each timed call,
 * "cK" = candidate K, and the chosen candidate
 * after "->"; candidates: c0 the split form whose scatter sums the lanes of one
 * grid cell in chunks of four, c1 the split form summing whole runs of such
 * lanes, c2 c3 the fused kernel in one wave / with 16 tiles per CTA, c4 c5 as
 * c0 c1 with the sampling-encoding kernel at 3 instead of 4 CTAs per SM; with
 * PRENOM_FLAG_FUSED: the fused kernel in one wave / 16 / 8 / 4 tiles per CTA;
 * PRENOM_FLAG_SPLIT: c0 untuned); then one line per step signature of
 * several groups: "step <its groups' signatures>:" with the whole-step times
 * of each round one after the other ("serial=") and forked ("forked="), and
 * the choice after "=>".  buf: host, cap bytes, NUL-terminated, truncated to
 * fit. */
PRENOM_API int prenom_tuning_report(prenom_ctx *ctx, char *buf, size_t cap);

/* Zeroes an object's gradient buffer (stream-ordered). */
PRENOM_API int prenom_zero_grads(prenom_ctx *ctx, int32_t obj);

/* Waits for the context's stream; returns the first asynchronous error, or
 * PRENOM_ERR_DEVICE_TIMEOUT (a bounded device wait gave up) or
 * PRENOM_ERR_DEVICE_BOUNDS (debug build only) from the device status word,
 * which it then clears. */
PRENOM_API int prenom_sync(prenom_ctx *ctx);

/* Kernel timing: when enabled, every library launch is bracketed by CUDA
 * events on the context's stream.  prenom_kernel_time() synchronises and
 * returns, for kernel id k (PRENOM_KERNEL_*), the summed device time in ms
 * and the launch count since timing was last enabled or reset. */
PRENOM_API int prenom_enable_timing(prenom_ctx *ctx, int32_t enable);
PRENOM_API int prenom_kernel_time(prenom_ctx *ctx, int32_t kernel, double *total_ms, int64_t *launches);

/* ------------------------------------------------- allocation-free step
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory when they train: a mapping front end
 * that reserved the GPU's whole memory budget for its own buffers up front, a
 * host framework whose caching allocator owns the device pool, or a real-time
 * thread that cannot afford cudaMalloc's implicit device synchronisation.
 *
 * prenom_train_step_noalloc() runs the training step of prenom_train_step()
 * (one batch, sampling through Adam) for one FP32 object whose state the
 * caller owns, in the fused FP32 kernel, and calls no cudaMalloc, cudaFree or
 * other allocating routine.  Its only extra device memory is a gradient
 * accumulator of PRENOM_NOALLOC_MAX_PARAMS floats (16 MiB) compiled into the
 * library as a static device array, which every GPU that loads the library
 * holds until the process exits.
 *   arch       architecture (same rules as prenom_create_object) with
 *              precision PRENOM_PRECISION_FP32 only (mixed-precision objects
 *              are rejected); objects with more than PRENOM_NOALLOC_MAX_PARAMS
 *              parameters are rejected; both with PRENOM_ERR_INVALID_ARG
 *   theta      device, param_count floats, updated in place (layout above)
 *   adam_m, adam_v  device, param_count floats each, updated in place (zero
 *              before the first step)
 *              theta, adam_m and adam_v must each be 16-byte aligned, else
 *              PRENOM_ERR_INVALID_ARG (checked on the host, nothing launched)
 *   step       Adam steps already taken (this call performs step + 1)
 *   grid, res  prior density grid as in prenom_set_prior_grid (device,
 *              2 <= res <= 1024; may be NULL when the batch gives t_in)
 *   batch      rays as for prenom_train_step (batch->obj only keys the Philox
 *              draws when uniforms or c_rand are NULL)
 *   opts       as for prenom_train_step; flags may hold only PRENOM_FLAG_FUSED
 *              and PRENOM_FLAG_NO_GRAPH (the call is always one fused launch
 *              and one Adam launch, never a graph); PRENOM_FLAG_NO_ADAM,
 *              PRENOM_FLAG_CHECK_FINITE and PRENOM_FLAG_SPLIT are refused with
 *              PRENOM_ERR_INVALID_ARG, since the gradient lives in the shared
 *              array only for the duration of one call
 *   loss_dev   device float receiving the batch's loss, or NULL
 *   cuda_stream, seed  stream of all work; Philox seed
 * Errors are reported by the return code; the message is available from
 * prenom_last_error(NULL).
 * The first call on each device looks up the array's device address (set-up
 * done once per device, with that device current); under CUDA's lazy module
 * loading that lookup is also what loads the library module holding the
 * array, so the first call may allocate the array and synchronise the device
 * inside the driver: make that first call during set-up, before any stream
 * capture and outside any section that must not allocate.  Every call on a
 * device shares the array and clears the part it uses before use, so calls
 * whose work overlaps on the GPU (for example on two streams at once) race
 * and must be avoided. */
#define PRENOM_NOALLOC_MAX_PARAMS (1 << 22)

PRENOM_API int prenom_train_step_noalloc(const prenom_arch *arch, float *theta, float *adam_m, float *adam_v,
                                         int32_t step, const float *grid, int32_t res,
                                         const prenom_ray_batch *batch, const prenom_train_opts *opts,
                                         float *loss_dev, void *cuda_stream, uint64_t seed);

/* Loss-scaling state of a mixed-precision object (blocking read): the current
 * scale and the number of steps dropped because a scaled 16-bit gradient
 * overflowed.  FP32 objects report scale 1 and 0 dropped steps. */
PRENOM_API int prenom_get_loss_scale(prenom_ctx *ctx, int32_t obj, float *scale, int32_t *dropped_steps);

/* Sets the loss scale of a mixed-precision object (1 <= scale <= 2^24) and the
 * number of clean steps in a row after which it doubles (growth_interval >= 1;
 * 1000 by default); the count of clean steps restarts at 0.  Blocking.  FP32
 * objects have no loss scale: PRENOM_ERR_INVALID_ARG. */
PRENOM_API int prenom_set_loss_scale(prenom_ctx *ctx, int32_t obj, float scale, int32_t growth_interval);

/* Total kernel launches made by the library on this context. */
PRENOM_API int prenom_launch_count(prenom_ctx *ctx, int64_t *launches);

#ifdef __cplusplus
}
#endif
#endif /* PRENOM_H */
