// Training step that allocates no device memory.
//
// Some callers cannot call cudaMalloc when they want to train: a mapping
// front end that reserved the whole GPU memory budget for its own keyframe
// and map buffers up front, a host framework whose caching allocator owns the
// device pool, or a real-time tracking thread that must not pay cudaMalloc's
// implicit device synchronisation in the middle of a frame.  They own theta
// and the Adam moments themselves and call prenom_train_step_noalloc(); the
// only extra device memory it uses is the gradient accumulator below, a
// fixed-size array that is part of the loaded library.
#include <math.h>
#include <stdio.h>

#include "prenom.h"
#include "prenom_internal.h"

namespace prenom {
int describe_caller_field(const prenom_arch *arch, const float *theta, float *grad, const float *grid, int32_t R,
                          ObjDesc *od, int64_t *n_params);
int check_caller_opts(const prenom_train_opts *op);
int set_context_free_error(int code, const char *msg);
}  // namespace prenom

using namespace prenom;

namespace {

constexpr int kMaxDevices = 64;

// Gradient accumulator (PRENOM_NOALLOC_MAX_PARAMS floats) plus one loss slot,
// shared by every call on a device; every GPU that loads the library holds it
// (16 MiB) until the process exits.
static __device__ __align__(256) float g_noalloc_scratch[PRENOM_NOALLOC_MAX_PARAMS + 64];

// Device address of g_noalloc_scratch per device (host code cannot use the
// symbol's name as an address).
float *g_scratch_addr[kMaxDevices] = {};

int err(int code, const char *fmt, long long a = 0, long long b = 0)
{
    char buf[256];
    snprintf(buf, sizeof(buf), fmt, a, b);
    return set_context_free_error(code, buf);
}

}  // namespace

extern "C" int prenom_train_step_noalloc(const prenom_arch *arch, float *theta, float *adam_m, float *adam_v,
                                         int32_t step, const float *grid, int32_t res, const prenom_ray_batch *batch,
                                         const prenom_train_opts *opts, float *loss_dev, void *cuda_stream,
                                         uint64_t seed)
{
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (!theta || !adam_m || !adam_v || !batch || !opts)
        return err(PRENOM_ERR_INVALID_ARG, "noalloc step: theta, adam_m, adam_v, batch and opts are required");
    // the Adam kernel reads and writes theta, m and v four floats at a time
    if (reinterpret_cast<uintptr_t>(theta) % 16 != 0 || reinterpret_cast<uintptr_t>(adam_m) % 16 != 0 ||
        reinterpret_cast<uintptr_t>(adam_v) % 16 != 0)
        return err(PRENOM_ERR_INVALID_ARG, "noalloc step: theta, adam_m and adam_v must be 16-byte aligned");
    if (step < 0)
        return err(PRENOM_ERR_INVALID_ARG, "noalloc step: step %lld < 0", step);
    int rc = check_caller_opts(opts);
    if (rc)
        return rc;
    // the gradient lives in the shared array only for the call, so it cannot be
    // accumulated over calls (NO_ADAM) and no per-call finiteness check exists
    if (opts->flags & ~(uint32_t)(PRENOM_FLAG_FUSED | PRENOM_FLAG_NO_GRAPH))
        return err(PRENOM_ERR_INVALID_ARG,
                   "noalloc step: flags 0x%llx not supported (only PRENOM_FLAG_FUSED and PRENOM_FLAG_NO_GRAPH)",
                   (long long)opts->flags);
    const prenom_ray_batch &b = *batch;
    if (b.n_rays < 0)
        return err(PRENOM_ERR_INVALID_ARG, "noalloc step: n_rays = %lld < 0", b.n_rays);
    if (b.n_rays > 0 && (!b.o || !b.d || !b.rgb || !b.depth || !b.is_obj))
        return err(PRENOM_ERR_INVALID_ARG, "noalloc step: o, d, rgb, depth and is_obj are required");
    if (b.n_rays > 0 && !b.t_in && !grid)
        return err(PRENOM_ERR_INVALID_ARG, "noalloc step: a prior grid is required without t_in");
    if (grid && (res < 2 || res > 1024))
        return err(PRENOM_ERR_INVALID_ARG, "noalloc step: res = %lld, must be 2..1024", res);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return err(PRENOM_ERR_CUDA, "noalloc step: no usable current device (device %lld)", dev);

    // One-time set-up per device (must happen outside stream capture).
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return err(PRENOM_ERR_CUDA, "noalloc step: cudaGetSymbolAddress failed (error %lld)", (long long)e);
        g_scratch_addr[dev] = static_cast<float *>(p);
    }
    float *grad = g_scratch_addr[dev];
    float *loss = loss_dev ? loss_dev : grad + PRENOM_NOALLOC_MAX_PARAMS;

    ObjDesc od;
    int64_t n = 0;
    rc = describe_caller_field(arch, theta, grad, grid, res, &od, &n);
    if (rc)
        return rc;
    if (arch->precision != PRENOM_PRECISION_FP32)
        return err(PRENOM_ERR_INVALID_ARG, "noalloc step: only FP32 objects (precision %lld given)", arch->precision);
    if (n > PRENOM_NOALLOC_MAX_PARAMS)
        return err(PRENOM_ERR_INVALID_ARG,
                   "noalloc step: the object has %lld parameters; the allocation-free step holds at most %lld", n,
                   (long long)PRENOM_NOALLOC_MAX_PARAMS);

    int n_sm = 0, optin = 0;
    e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess)
        return err(PRENOM_ERR_CUDA, "noalloc step: device query failed (error %lld)", (long long)e);

    // The array keeps the previous call's contents: clear the gradient and the loss.
    e = cudaMemsetAsync(grad, 0, (size_t)n * sizeof(float), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e != cudaSuccess)
        return err(PRENOM_ERR_CUDA, "noalloc step: clearing the scratch failed (error %lld)", (long long)e);

    if (b.n_rays > 0) {
        const int S = fused_fp32_pick_tile(od.W, od.IN, od.H, (size_t)optin);
        if (S == 0)
            return err(PRENOM_ERR_INVALID_ARG, "noalloc step: the architecture does not fit in shared memory");
        if (opts->nr > S)
            return err(PRENOM_ERR_INVALID_ARG, "noalloc step: nr = %lld exceeds the %lld-sample tile of this architecture",
                       (long long)opts->nr, (long long)S);
        BatchDesc bd{};
        bd.n_rays = b.n_rays;
        bd.nc = opts->nc;
        bd.nr = opts->nr;
        bd.rays_per_tile = S / opts->nr;
        bd.n_tiles = (b.n_rays + bd.rays_per_tile - 1) / bd.rays_per_tile;
        bd.mode = kTrain;
        bd.escape_eps = opts->escape_eps;
        bd.inv_r = 1.f / (float)b.n_rays;
        bd.o = b.o;
        bd.d = b.d;
        bd.rgb = b.rgb;
        bd.depth = b.depth;
        bd.is_obj = b.is_obj;
        bd.c_rand = b.c_rand;
        bd.u = b.uniforms;
        bd.t_in = b.t_in;
        bd.loss = loss;
        bd.seed = seed;
        bd.step = (uint32_t)step;
        bd.obj_id = (uint32_t)b.obj;
        e = launch_fused_fp32(od, bd, S, bd.n_tiles < n_sm ? bd.n_tiles : n_sm, st);
        if (e != cudaSuccess)
            return err(PRENOM_ERR_CUDA, "noalloc step: fused kernel launch failed (error %lld)", (long long)e);
    }

    AdamArgs a{};
    a.n_segs = 1;
    a.beta1 = opts->beta1;
    a.beta2 = opts->beta2;
    a.eps = opts->eps;
    const double t = (double)step + 1.0;
    a.seg[0].theta = theta;
    a.seg[0].grad = grad;
    a.seg[0].m = adam_m;
    a.seg[0].v = adam_v;
    a.seg[0].n = n;
    a.seg[0].lr_c1 = (float)((double)opts->lr / (1.0 - pow((double)opts->beta1, t)));
    a.seg[0].inv_c2 = (float)(1.0 / (1.0 - pow((double)opts->beta2, t)));
    a.chunk_start[0] = 0;
    a.chunk_start[1] = (n + kAdamChunk - 1) / kAdamChunk;
    const int64_t chunks = a.chunk_start[1];
    const int grid_adam = (int)(chunks < (int64_t)n_sm * 8 ? chunks : (int64_t)n_sm * 8);
    if (grid_adam > 0) {
        e = launch_adam(a, grid_adam, st);
        if (e != cudaSuccess)
            return err(PRENOM_ERR_CUDA, "noalloc step: Adam launch failed (error %lld)", (long long)e);
    }
    return PRENOM_OK;
}
