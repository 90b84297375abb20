// C ABI of the PRENOM training library: object registry, device arenas,
// argument checking, launch configuration, Adam bookkeeping and kernel timing.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <set>
#include <new>
#include <string>
#include <vector>

#include "prenom.h"
#include "prenom_internal.h"

using namespace prenom;

namespace {

std::string g_create_error;
constexpr int kScratchLosses = 64;  // device floats of prenom_ctx::scratch

struct Object {
    bool alive = false;
    prenom_arch arch{};
    int IN = 0;
    int64_t n = 0, n_hash = 0, n_pad = 0;
    std::vector<int32_t> res, dense;
    std::vector<int64_t> off;  // float offsets, L + 1 entries
    float *arena = nullptr, *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    uint16_t *feat16 = nullptr;  // BF16 copy of the hash tables (PRENOM_FEATURES_BF16)
    float *grid = nullptr;
    int32_t R = 0;
    int32_t step = 0;
    LossScaleState *lss = nullptr;  // mixed precision only
};

struct TimedEv {
    cudaEvent_t a, b;
    int kernel;
    int group;  // index into prenom_ctx::group_names, or -1 outside a batched group
};

}  // namespace

struct prenom_ctx {
    cudaStream_t stream = nullptr;
    uint64_t seed = 0;
    int device = 0, n_sm = 0;
    size_t smem_optin = 0;
    std::vector<Object> objs;
    std::string err;
    float *scratch = nullptr;  // device float receiving losses nobody asked for
    int32_t *status = nullptr; // device word: kStatusWait (a bounded wait gave up), kStatusBounds (debug build)
    bool timing = false;
    std::vector<TimedEv> pending;
    std::vector<cudaEvent_t> ev_free;
    double total_ms[PRENOM_N_KERNELS] = {};
    int64_t count[PRENOM_N_KERNELS] = {};
    int64_t launches = 0;
    // timed batched steps: kernel times per (group, kernel id)
    int cur_group = -1;
    std::vector<std::string> group_names;
    std::map<std::pair<int, int>, std::pair<double, int64_t>> group_time;
    mutable std::map<int, int> tc_occ;  // resident tensor-core CTAs per SM by variant
    int64_t n_captures = 0;    // step graphs captured
    int64_t n_tune_calls = 0;  // steps run as autotuner measurements
    // batched steps: device work list (+ per-object Adam factors behind it),
    // two pinned staging buffers, the graphs captured per step signature and
    // the autotuner's choice of tiles per CTA per group signature
    unsigned char *d_work = nullptr;
    size_t d_work_cap = 0;
    unsigned char *h_stage[2] = {nullptr, nullptr};
    size_t h_stage_cap = 0;
    cudaEvent_t stage_ev[2] = {nullptr, nullptr};
    int stage_idx = 0;
    // the groups of a batched step after the first run on streams of their own,
    // forked from the context's stream and joined back before Adam
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> side_ev;  // [0] the fork, [1 + i] the join of side stream i
    struct CachedGraph {
        cudaGraphExec_t exec;
        uint64_t last_use;
    };
    std::map<std::string, CachedGraph> graphs;  // at most kMaxGraphs, least recently used evicted
    uint64_t graph_tick = 0;
    std::map<std::string, std::vector<float>> tune_ms;  // measured ms per candidate
    std::map<std::string, int> tune_best;               // chosen candidate index
    std::set<std::string> tune_warm;                    // signatures past their untimed first call
    // per step signature (its groups' signatures): whole-step times one after the
    // other and forked ([2 q] and [2 q + 1] of round q), and the choice
    std::map<std::string, std::vector<float>> fork_ms;
    std::map<std::string, bool> fork_best;
    // split form of mixed-precision training: the buffers its kernels hand over
    unsigned char *split_buf = nullptr;
    size_t split_cap = 0;
    // density-grid queries and yaw scores
    unsigned char *query_buf = nullptr;
    size_t query_cap = 0;
    // training-ray generation
    unsigned char *rays_buf = nullptr;
    size_t rays_cap = 0;
    uint32_t ray_calls = 0;
};

namespace {

int fail(prenom_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_create_error = buf;
    return code;
}

int cuda_fail(prenom_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, PRENOM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Level resolutions of the multiresolution grid (instant-NGP, cited in §III-B):
// N_l = floor(N_min b^l) with b = exp((ln N_max - ln N_min) / (L - 1)), a 1e-6
// guard keeping mathematically integral products from rounding down; a level
// is dense when its (N_l + 1)^3 vertices fit in T entries.
void level_geometry(const prenom_arch &a, Object &o)
{
    const double b = a.L > 1 ? exp((log((double)a.n_max) - log((double)a.n_min)) / (double)(a.L - 1)) : 1.0;
    const int64_t T = (int64_t)1 << a.log2T;
    o.res.assign(a.L, 0);
    o.dense.assign(a.L, 0);
    o.off.assign(a.L + 1, 0);
    for (int l = 0; l < a.L; ++l) {
        const int N = (int)floor((double)a.n_min * pow(b, (double)l) + 1e-6);
        const int64_t v = (int64_t)(N + 1) * (N + 1) * (N + 1);
        o.res[l] = N;
        o.dense[l] = v <= T;
        // each level padded to a multiple of 8 entries: levels start 64-byte
        // aligned, so an aligned pair of entries is one 16-byte access
        o.off[l + 1] = o.off[l] + ((o.dense[l] ? v : T) + 7) / 8 * 8 * a.F;
    }
    o.n_hash = o.off[a.L];
    o.IN = a.L * a.F;
    o.n = o.n_hash + (int64_t)a.width * o.IN + (int64_t)(a.hidden - 1) * a.width * a.width + 4LL * a.width;
    o.n_pad = (o.n + 63) / 64 * 64;
}

int check_arch(prenom_ctx *c, const prenom_arch *a)
{
    if (!a)
        return fail(c, PRENOM_ERR_INVALID_ARG, "arch is NULL");
    if (a->F != 2)
        return fail(c, PRENOM_ERR_INVALID_ARG, "F = %d: this build supports F = 2", a->F);
    if (a->L != 4 && a->L != 8 && a->L != 16)
        return fail(c, PRENOM_ERR_INVALID_ARG, "L = %d: this build supports L in {4, 8, 16}", a->L);
    if (a->width != 16 && a->width != 32 && a->width != 64)
        return fail(c, PRENOM_ERR_INVALID_ARG, "width = %d: must be 16, 32 or 64", a->width);
    if (a->hidden < 1 || a->hidden > kMaxHidden)
        return fail(c, PRENOM_ERR_INVALID_ARG, "hidden = %d: must be 1..%d", a->hidden, kMaxHidden);
    if (a->log2T < 8 || a->log2T > 24)
        return fail(c, PRENOM_ERR_INVALID_ARG, "log2T = %d: must be 8..24", a->log2T);
    if (a->n_min < 2 || a->n_max < a->n_min || a->n_max > (1 << 20))
        return fail(c, PRENOM_ERR_INVALID_ARG, "resolutions %d..%d out of range", a->n_min, a->n_max);
    if (a->precision != PRENOM_PRECISION_FP32 && a->precision != PRENOM_PRECISION_FP16 &&
        a->precision != PRENOM_PRECISION_BF16)
        return fail(c, PRENOM_ERR_INVALID_ARG, "precision %d: must be FP32 (0), FP16 (1) or BF16 (2)", a->precision);
    if (!(a->lambda_d >= 0.f) || !(a->lambda_sigma >= 0.f) || !isfinite(a->lambda_d) || !isfinite(a->lambda_sigma))
        return fail(c, PRENOM_ERR_INVALID_ARG, "lambda_d and lambda_sigma must be finite and >= 0");
    if (a->features != PRENOM_FEATURES_FP32 && a->features != PRENOM_FEATURES_BF16)
        return fail(c, PRENOM_ERR_INVALID_ARG, "features %d: must be FP32 (0) or BF16 (2)", a->features);
    if (a->features == PRENOM_FEATURES_BF16 && a->precision == PRENOM_PRECISION_FP32)
        return fail(c, PRENOM_ERR_INVALID_ARG, "BF16 features need a mixed-precision object");
    return PRENOM_OK;
}

Object *get_obj(prenom_ctx *c, int32_t obj)
{
    if (!c || obj < 0 || obj >= (int32_t)c->objs.size() || !c->objs[obj].alive)
        return nullptr;
    return &c->objs[obj];
}

int check_opts(prenom_ctx *c, const prenom_train_opts *op, bool need_adam)
{
    if (!op)
        return fail(c, PRENOM_ERR_INVALID_ARG, "opts is NULL");
    if (op->nr < kMinNr || op->nr > kMaxNr)
        return fail(c, PRENOM_ERR_INVALID_ARG, "nr = %d: must be %d..%d", op->nr, kMinNr, kMaxNr);
    if (op->nc < 1 || op->nc > kMaxNc)
        return fail(c, PRENOM_ERR_INVALID_ARG, "nc = %d: must be 1..%d", op->nc, kMaxNc);
    if (!(op->escape_eps >= 0.f) || !isfinite(op->escape_eps))
        return fail(c, PRENOM_ERR_INVALID_ARG, "escape_eps must be finite and >= 0");
    if (!(op->loss_scale_init >= 0.f) || !isfinite(op->loss_scale_init))
        return fail(c, PRENOM_ERR_INVALID_ARG, "loss_scale_init must be finite and >= 0");
    if (need_adam && !(op->flags & PRENOM_FLAG_NO_ADAM)) {
        if (!isfinite(op->lr) || !(op->beta1 >= 0.f && op->beta1 < 1.f) || !(op->beta2 >= 0.f && op->beta2 < 1.f) ||
            !(op->eps >= 0.f) || !isfinite(op->eps))
            return fail(c, PRENOM_ERR_INVALID_ARG, "Adam constants out of range");
    }
    return PRENOM_OK;
}

int check_batch(prenom_ctx *c, const prenom_ray_batch &b, bool train)
{
    Object *o = get_obj(c, b.obj);
    if (!o)
        return fail(c, PRENOM_ERR_INVALID_ARG, "batch names unknown object %d", b.obj);
    if (b.n_rays < 0)
        return fail(c, PRENOM_ERR_INVALID_ARG, "n_rays = %d < 0", b.n_rays);
    if (b.n_rays == 0)
        return PRENOM_OK;
    if (!b.o || !b.d)
        return fail(c, PRENOM_ERR_INVALID_ARG, "ray origins and directions are required");
    if (train && (!b.rgb || !b.depth || !b.is_obj))
        return fail(c, PRENOM_ERR_INVALID_ARG, "training needs rgb, depth and is_obj");
    if (!b.t_in && !o->grid)
        return fail(c, PRENOM_ERR_INVALID_ARG, "object %d has no prior grid and the batch gives no t_in", b.obj);
    return PRENOM_OK;
}

void timed_begin(prenom_ctx *c, int kernel, cudaEvent_t *a)
{
    *a = nullptr;
    if (!c->timing)
        return;
    if (c->ev_free.empty()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev_free.push_back(e);
    }
    *a = c->ev_free.back();
    c->ev_free.pop_back();
    cudaEventRecord(*a, c->stream);
    (void)kernel;
}

void timed_end(prenom_ctx *c, int kernel, cudaEvent_t a)
{
    c->launches++;
    if (!c->timing || !a)
        return;
    if (c->ev_free.empty()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->ev_free.push_back(e);
    }
    cudaEvent_t b = c->ev_free.back();
    c->ev_free.pop_back();
    cudaEventRecord(b, c->stream);
    c->pending.push_back({a, b, kernel, c->cur_group});
}

// Adds the durations of all recorded event pairs to the totals (after the stream finished).
void fold_pending(prenom_ctx *c)
{
    for (auto &p : c->pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.a, p.b);
        c->total_ms[p.kernel] += ms;
        c->count[p.kernel] += 1;
        if (p.group >= 0) {
            auto &g = c->group_time[{p.group, p.kernel}];
            g.first += ms;
            g.second += 1;
        }
        c->ev_free.push_back(p.a);
        c->ev_free.push_back(p.b);
    }
    c->pending.clear();
}

ObjDesc make_objdesc(const Object &o, float *grad)
{
    ObjDesc d{};
    d.theta = o.theta;
    d.feat16 = reinterpret_cast<const uint32_t *>(o.feat16);
    d.grad = grad;
    d.L = o.arch.L;
    d.IN = o.IN;
    d.W = o.arch.width;
    d.H = o.arch.hidden;
    d.tmask = (uint32_t)((1u << o.arch.log2T) - 1u);
    d.mlp_off = (uint32_t)o.n_hash;
    for (int l = 0; l < o.arch.L; ++l) {
        d.lv[l].res = o.res[l];
        d.lv[l].offset = (uint32_t)(o.off[l] / o.arch.F);
        d.lv[l].dense = o.dense[l];
    }
    d.grid = o.grid;
    d.R = o.R;
    d.lambda_d = o.arch.lambda_d;
    d.lambda_sigma = o.arch.lambda_sigma;
    return d;
}

BatchDesc make_batchdesc(const prenom_ctx *c, const Object &o, const prenom_ray_batch &b, const prenom_train_opts &op,
                         int mode, int S)
{
    BatchDesc d{};
    d.n_rays = b.n_rays;
    d.nc = op.nc;
    d.nr = op.nr;
    d.rays_per_tile = S / op.nr;
    d.n_tiles = (b.n_rays + d.rays_per_tile - 1) / d.rays_per_tile;
    d.mode = mode;
    d.escape_eps = op.escape_eps;
    d.inv_r = b.n_rays > 0 ? 1.f / (float)b.n_rays : 0.f;
    d.o = b.o;
    d.d = b.d;
    d.rgb = b.rgb;
    d.depth = b.depth;
    d.is_obj = b.is_obj;
    d.c_rand = b.c_rand;
    d.u = b.uniforms;
    d.t_in = b.t_in;
    d.seed = c->seed;
    d.step = (uint32_t)o.step;
    d.obj_id = (uint32_t)b.obj;
    if (o.lss && mode == kTrain) {
        d.loss_scale = &o.lss->scale;
        d.overflow = &o.lss->overflow;
    }
    if (o.lss && o.arch.precision == PRENOM_PRECISION_FP16)
        d.enc_scale = &o.lss->enc_scale;
    d.status = c->status;
    return d;
}

// Grows the split-form buffer to at least `bytes` (waits for the stream first:
// the previous step may still read the old buffer).
int ensure_split(prenom_ctx *c, size_t bytes)
{
    if (bytes <= c->split_cap)
        return PRENOM_OK;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "stream");
    cudaFree(c->split_buf);
    c->split_buf = nullptr;
    c->split_cap = 0;
    const size_t cap = bytes + bytes / 4;
    e = cudaMalloc(&c->split_buf, cap);
    if (e != cudaSuccess)
        return fail(c, PRENOM_ERR_OOM, "split-form buffers of %zu bytes: %s", cap, cudaGetErrorString(e));
    c->split_cap = cap;
    return PRENOM_OK;
}

// Points a batch's split buffers into base; returns the bytes they take.
size_t assign_split(BatchDesc &bd, unsigned char *base)
{
    const size_t t_bytes = ((size_t)bd.n_rays * bd.nr * sizeof(float) + 255) / 256 * 256;
    bd.sp_t = reinterpret_cast<float *>(base);
    bd.sp_x = reinterpret_cast<uint4 *>(base + t_bytes);
    bd.sp_dx = reinterpret_cast<float2 *>(base + t_bytes + (size_t)bd.n_tiles * kSplitXBytes);
    bd.sp_rays = reinterpret_cast<float *>(base + t_bytes + (size_t)bd.n_tiles * (kSplitXBytes + kSplitDx * 8));
    return split_bytes(bd.n_rays, bd.nr, bd.n_tiles);
}

// Grids of the split form's two extra kernels: the sampling-encoding kernel
// runs one warp per ray slot with per_sm (4 or 3) CTAs per SM, the scatter
// kernel one block per tile range.
int grid_sample_encode(const prenom_ctx *c, int total_tiles, int rays_per_tile, int per_sm = 4)
{
    const int64_t slots = (int64_t)total_tiles * rays_per_tile;  // one block per slot at most
    return (int)std::max<int64_t>(1, std::min<int64_t>(slots, (int64_t)c->n_sm * per_sm));
}

int grid_scatter(const prenom_ctx *c, int total_tiles)
{
    return std::max(1, std::min(total_tiles, c->n_sm * 5));  // five 256-thread CTAs per SM (48 registers)
}

// Resident CTAs per SM of a tensor-core kernel variant (queried once per variant).
int tc_per_sm(const prenom_ctx *c, int precision, int W, int IN, int H, bool split)
{
    const int key = (((precision * 128 + W) * 64 + IN) * 8 + H) * 2 + (split ? 1 : 0);
    auto it = c->tc_occ.find(key);
    if (it != c->tc_occ.end())
        return it->second;
    const int n = fused_tc_occupancy(precision, W, IN, H, split);
    c->tc_occ[key] = n;
    return n;
}

int launch_fused(prenom_ctx *c, const Object &o, const ObjDesc &od, BatchDesc &bd, int kernel_id, bool split = false)
{
    if (bd.n_rays == 0)
        return PRENOM_OK;
    if (o.arch.precision != PRENOM_PRECISION_FP32) {
        const size_t smem = fused_tc_smem(od.W, od.IN, od.H, split && bd.mode == kTrain);
        if (smem == 0 || smem > c->smem_optin)
            return fail(c, PRENOM_ERR_INVALID_ARG, "architecture needs more shared memory than the device offers");
        bd.rays_per_tile = 128 / bd.nr;
        bd.n_tiles = (bd.n_rays + bd.rays_per_tile - 1) / bd.rays_per_tile;
        const int per_sm = std::max(1, tc_per_sm(c, o.arch.precision, od.W, od.IN, od.H, split && bd.mode == kTrain));
        const int grid = std::min(bd.n_tiles, c->n_sm * per_sm);
        if (split && bd.mode == kTrain) {
            int rc = ensure_split(c, split_bytes(bd.n_rays, bd.nr, bd.n_tiles));
            if (rc)
                return rc;
            assign_split(bd, c->split_buf);
            WorkItem one{};
            one.od = od;
            one.bd = bd;
            const WorkList wl{nullptr, 1, bd.n_tiles, od.H, 1, od.feat16 != nullptr};
            cudaEvent_t ev;
            timed_begin(c, PRENOM_KERNEL_SAMPLE_ENCODE, &ev);
            cudaError_t e = launch_sample_encode(one, wl, o.arch.precision, 4,
                                                 grid_sample_encode(c, bd.n_tiles, bd.rays_per_tile), c->stream);
            timed_end(c, PRENOM_KERNEL_SAMPLE_ENCODE, ev);
            if (e != cudaSuccess)
                return cuda_fail(c, e, "sampling-encoding kernel launch");
            timed_begin(c, kernel_id, &ev);
            e = launch_fused_tc(od, bd, o.arch.precision, grid, c->stream);
            timed_end(c, kernel_id, ev);
            if (e != cudaSuccess)
                return cuda_fail(c, e, "mixed-precision kernel launch");
            timed_begin(c, PRENOM_KERNEL_SCATTER, &ev);
            e = launch_hash_scatter(one, wl, grid_scatter(c, bd.n_tiles), c->stream);
            timed_end(c, PRENOM_KERNEL_SCATTER, ev);
            if (e != cudaSuccess)
                return cuda_fail(c, e, "hash scatter kernel launch");
            return PRENOM_OK;
        }
        cudaEvent_t ev;
        timed_begin(c, kernel_id, &ev);
        const cudaError_t e = launch_fused_tc(od, bd, o.arch.precision, grid, c->stream);
        timed_end(c, kernel_id, ev);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "mixed-precision kernel launch");
        return PRENOM_OK;
    }
    const int S = fused_fp32_pick_tile(od.W, od.IN, od.H, c->smem_optin);
    if (S == 0)
        return fail(c, PRENOM_ERR_INVALID_ARG, "architecture needs more shared memory than the device offers");
    if (bd.nr > S)
        return fail(c, PRENOM_ERR_INVALID_ARG, "nr = %d exceeds the %d-sample tile of this architecture", bd.nr, S);
    bd.rays_per_tile = S / bd.nr;
    bd.n_tiles = (bd.n_rays + bd.rays_per_tile - 1) / bd.rays_per_tile;
    const int grid = std::min(bd.n_tiles, c->n_sm);
    if (split && bd.mode == kTrain) {
        int rc = ensure_split(c, split_bytes(bd.n_rays, bd.nr, bd.n_tiles));
        if (rc)
            return rc;
        assign_split(bd, c->split_buf);
        WorkItem one{};
        one.od = od;
        one.bd = bd;
        const WorkList wl{nullptr, 1, bd.n_tiles, od.H, 1};
        cudaEvent_t ev;
        timed_begin(c, PRENOM_KERNEL_SAMPLE_ENCODE, &ev);
        cudaError_t e = launch_sample_encode(one, wl, PRENOM_PRECISION_FP32, 4,
                                             grid_sample_encode(c, bd.n_tiles, bd.rays_per_tile), c->stream);
        timed_end(c, PRENOM_KERNEL_SAMPLE_ENCODE, ev);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "sampling-encoding kernel launch");
        timed_begin(c, kernel_id, &ev);
        e = launch_fused_fp32(od, bd, S, grid, c->stream);
        timed_end(c, kernel_id, ev);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "fused kernel launch");
        timed_begin(c, PRENOM_KERNEL_SCATTER, &ev);
        e = launch_hash_scatter(one, wl, grid_scatter(c, bd.n_tiles), c->stream);
        timed_end(c, PRENOM_KERNEL_SCATTER, ev);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "hash scatter kernel launch");
        return PRENOM_OK;
    }
    cudaEvent_t ev;
    timed_begin(c, kernel_id, &ev);
    const cudaError_t e = launch_fused_fp32(od, bd, S, grid, c->stream);
    timed_end(c, kernel_id, ev);
    (void)o;
    if (e != cudaSuccess)
        return cuda_fail(c, e, "fused kernel launch");
    return PRENOM_OK;
}

// Where Adam gathers max |hash entry| of an FP16 object (its encoding scale follows it).
uint32_t *enc_absmax_ptr(const Object &o)
{
    return o.lss && o.arch.precision == PRENOM_PRECISION_FP16 ? &o.lss->hash_absmax : nullptr;
}

// Recomputes what an object derives from its hash tables -- the BF16 copy the
// gathers read and an FP16 object's encoding scale -- after a write of theta
// that Adam did not make.
int refresh_enc_scale(prenom_ctx *c, const Object &o)
{
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((o.n_hash + 1023) / 1024, (int64_t)c->n_sm * 8));
    cudaError_t e = cudaSuccess;
    if (o.feat16) {
        e = launch_mirror_refresh(o.theta, o.n_hash, o.feat16, grid, c->stream);
        c->launches += 1;
    }
    if (e == cudaSuccess && enc_absmax_ptr(o)) {
        e = launch_enc_scale_refresh(o.theta, o.n_hash, o.lss, grid, c->stream);
        c->launches += 2;
    }
    return e == cudaSuccess ? PRENOM_OK : cuda_fail(c, e, "refresh of the tables' copy and scale");
}

int run_adam(prenom_ctx *c, const std::vector<int32_t> &objs, const prenom_train_opts &op)
{
    for (size_t first = 0; first < objs.size(); first += kMaxAdamSegs) {
        AdamArgs a{};
        a.beta1 = op.beta1;
        a.beta2 = op.beta2;
        a.eps = op.eps;
        const size_t last = std::min(objs.size(), first + kMaxAdamSegs);
        a.n_segs = (int32_t)(last - first);
        a.chunk_start[0] = 0;
        for (size_t i = first; i < last; ++i) {
            Object &o = c->objs[objs[i]];
            o.step += 1;
            const double c1 = 1.0 - pow((double)op.beta1, (double)o.step);
            const double c2 = 1.0 - pow((double)op.beta2, (double)o.step);
            AdamSeg &s = a.seg[i - first];
            s.theta = o.theta;
            s.grad = o.grad;
            s.m = o.m;
            s.v = o.v;
            s.n = o.n;
            s.lr_c1 = (float)((double)op.lr / c1);
            s.inv_c2 = (float)(1.0 / c2);
            s.skip = o.lss ? &o.lss->overflow : nullptr;
            s.absmax = enc_absmax_ptr(o);
            s.n_hash = o.n_hash;
            s.mirror = o.feat16;
            a.chunk_start[i - first + 1] = a.chunk_start[i - first] + (o.n + kAdamChunk - 1) / kAdamChunk;
        }
        const int64_t chunks = a.chunk_start[a.n_segs];
        const int grid = (int)std::min<int64_t>(chunks, (int64_t)c->n_sm * 16);
        if (grid == 0)
            continue;
        cudaEvent_t ev;
        timed_begin(c, PRENOM_KERNEL_ADAM, &ev);
        const cudaError_t e = launch_adam(a, grid, c->stream);
        timed_end(c, PRENOM_KERNEL_ADAM, ev);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "Adam launch");
        for (size_t i = first; i < last; ++i) {
            Object &o = c->objs[objs[i]];
            if (!o.lss)
                continue;
            const cudaError_t e2 = launch_loss_scale_update(o.lss, c->stream);
            c->launches++;
            if (e2 != cudaSuccess)
                return cuda_fail(c, e2, "loss-scale update launch");
        }
    }
    return PRENOM_OK;
}

// ------------------------------------------------------------ batched step
// A batched step groups its (object, batch) items by kernel variant
// (precision, W, IN, tile) and runs each group as one persistent launch over
// a device work list; one Adam launch then updates every object.  The work
// list and the per-object Adam factors are copied from a pinned staging
// buffer by the step itself, so the whole step can be captured once per
// signature as a CUDA graph and replayed with new rays.
struct Group {
    int precision, W, IN, S, hmax, first, count, total_tiles, grid;
    bool split = false;  // mixed precision: the three-kernel split form
    bool whole_runs = false;  // split form: the scatter sums whole runs of lanes
    int enc_per_sm = 4;       // split form: resident CTAs per SM of the sampling-encoding kernel
    int feat16 = 0;      // the group's gathers read BF16 copies of the tables
};

struct Plan {
    std::vector<WorkItem> items;
    std::vector<Group> groups;
    std::vector<int32_t> touched;   // objects updated by Adam, first appearance order
    std::vector<float2> adam_scal;  // (lr_c1, inv_c2) per touched object
    AdamArgs adam{};                // constant across steps (factors read from device)
    int adam_grid = 0;
    // per group: its objects' segments of `adam` (indices into touched) and their
    // parameter count; a forked step runs each group's Adam on the group's stream
    std::vector<std::vector<int>> group_segs;
    std::vector<int64_t> group_params;
    ScaleList scales{};
};

// Candidates of the autotuner: tiles per CTA of the training kernel (0 = one
// persistent wave of resident CTAs).  A group tries the split form first (its
// MLP kernel in one wave), with the scatter summing lanes of one cell in chunks
// of four (c0) or over whole runs (c1), then the fused kernel in one wave (c2)
// and with 16 tiles per CTA (c3), then the split form again with the
// sampling-encoding kernel at 3 CTAs per SM instead of 4 (c4: chunks of four,
// c5: whole runs); with the split form excluded, the fused kernel with four
// work-chunk sizes.
constexpr int kTuneTpc[] = {0, 16, 8, 4};
constexpr int kTuneTpcTc[] = {0, 0, 0, 16, 0, 0};
constexpr int kTuneNSplit = 6, kTuneNFused = 4;
constexpr int kTuneRounds = 3;  // each candidate is timed this many times (one step each); the median counts
constexpr size_t kMaxGraphs = 64;  // captured step graphs kept per context

int tune_n(bool split_allowed) { return split_allowed ? kTuneNSplit : kTuneNFused; }

bool cand_split(const Group &, int cand, bool split_allowed)
{
    return split_allowed && (cand <= 1 || cand >= 4);
}

bool cand_whole_runs(int cand, bool split_allowed)
{
    return split_allowed && (cand == 1 || cand == 5);
}

int cand_enc_per_sm(int cand, bool split_allowed)
{
    return split_allowed && cand >= 4 ? 3 : 4;
}

int group_grid(const prenom_ctx *c, const Group &g, int cand, bool split_allowed)
{
    int per_sm = 1;
    if (g.precision != PRENOM_PRECISION_FP32)
        per_sm = std::max(1, tc_per_sm(c, g.precision, g.W, g.IN, g.hmax, cand_split(g, cand, split_allowed)));
    const int wave = c->n_sm * per_sm;
    const int tpc = split_allowed ? kTuneTpcTc[cand] : kTuneTpc[cand];
    if (tpc == 0)
        return std::max(1, std::min(g.total_tiles, wave));
    return std::max(1, std::min(g.total_tiles, std::max(wave, (g.total_tiles + tpc - 1) / tpc)));
}

std::string group_key(const Group &g)
{
    char buf[128];
    snprintf(buf, sizeof(buf), "%d/%d/%d/%d/%d/%d/%d/%d", g.precision, g.W, g.IN, g.S, g.hmax, g.count, g.total_tiles,
             g.feat16);
    return buf;
}

// The autotuner's signature of a group: the kernel variant and the sizes in
// powers of two, so that steps whose ray counts vary a little share one tuning.
std::string tune_key(const Group &g)
{
    auto lg = [](int x) { int b = 0; while (x > 1) { x >>= 1; ++b; } return b; };
    char buf[128];
    snprintf(buf, sizeof(buf), "%d/%d/%d/%d/%d/n%d/t%d%s", g.precision, g.W, g.IN, g.S, g.hmax, lg(g.count),
             lg(g.total_tiles), g.feat16 ? "/b" : "");
    return buf;
}

// A group as the timing report names it: precision, widths, deepest MLP, batch
// and tile counts, form and grid.
std::string group_label(const Group &g)
{
    static const char *prec[] = {"fp32", "fp16", "bf16"};
    char buf[160];
    const char *form = !g.split ? "fused"
                       : g.whole_runs ? (g.enc_per_sm == 3 ? "split-runs-enc3" : "split-runs")
                                      : (g.enc_per_sm == 3 ? "split-enc3" : "split");
    snprintf(buf, sizeof(buf), "%s W%d IN%d H%d batches%d tiles%d %s grid%d%s", prec[g.precision], g.W, g.IN, g.hmax,
             g.count, g.total_tiles, form, g.grid, g.feat16 ? " bf16-features" : "");
    return buf;
}

int group_index(prenom_ctx *c, const std::string &label)
{
    for (size_t i = 0; i < c->group_names.size(); ++i)
        if (c->group_names[i] == label)
            return (int)i;
    c->group_names.push_back(label);
    return (int)c->group_names.size() - 1;
}

int plan_batched(prenom_ctx *c, const prenom_ray_batch *batches, int n, const prenom_train_opts &op, float *loss_dev,
                 Plan &p)
{
    std::vector<std::array<int, 5>> keys(n);
    for (int i = 0; i < n; ++i) {
        const Object &o = c->objs[batches[i].obj];
        int S = 128;
        if (o.arch.precision == PRENOM_PRECISION_FP32) {
            S = fused_fp32_pick_tile(o.arch.width, o.IN, o.arch.hidden, c->smem_optin);
            if (S == 0)
                return fail(c, PRENOM_ERR_INVALID_ARG, "architecture needs more shared memory than the device offers");
            if (op.nr > S)
                return fail(c, PRENOM_ERR_INVALID_ARG, "nr = %d exceeds the %d-sample tile of this architecture",
                            op.nr, S);
        }
        keys[i] = {o.arch.precision, o.arch.width, o.IN, S, o.arch.features == PRENOM_FEATURES_BF16 ? 1 : 0};
    }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i)
        order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return keys[a] < keys[b]; });
    p.items.resize(n);
    for (int j = 0; j < n;) {
        Group g{keys[order[j]][0], keys[order[j]][1], keys[order[j]][2], keys[order[j]][3], 1, j, 0, 0, 0};
        g.feat16 = keys[order[j]][4];
        int tiles = 0;
        while (j < n && keys[order[j]] == keys[order[g.first]]) {
            const int i = order[j];
            const prenom_ray_batch &b = batches[i];
            const Object &o = c->objs[b.obj];
            WorkItem &w = p.items[j];
            w.od = make_objdesc(o, o.grad);
            w.bd = make_batchdesc(c, o, b, op, kTrain, g.S);
            w.bd.loss = loss_dev ? loss_dev + i : c->scratch;
            w.tile_begin = tiles;
            tiles += w.bd.n_tiles;
            g.hmax = std::max(g.hmax, o.arch.hidden);
            ++g.count;
            ++j;
        }
        g.total_tiles = tiles;
        const size_t smem = g.precision == PRENOM_PRECISION_FP32 ? fused_fp32_smem(g.W, g.IN, g.hmax, g.S)
                                                                 : fused_tc_smem(g.W, g.IN, g.hmax, true);
        if (smem == 0 || smem > c->smem_optin)
            return fail(c, PRENOM_ERR_INVALID_ARG, "architecture group needs more shared memory than the device offers");
        p.groups.push_back(g);
    }
    for (int i = 0; i < n; ++i)
        if (std::find(p.touched.begin(), p.touched.end(), batches[i].obj) == p.touched.end())
            p.touched.push_back(batches[i].obj);
    for (const Group &g : p.groups) {  // an object's batches all fall in one group (its architecture's)
        std::vector<int> segs;
        int64_t params = 0;
        for (int j = g.first; j < g.first + g.count; ++j) {
            const int32_t obj = batches[order[j]].obj;
            const int s = (int)(std::find(p.touched.begin(), p.touched.end(), obj) - p.touched.begin());
            if (std::find(segs.begin(), segs.end(), s) == segs.end()) {
                segs.push_back(s);
                params += c->objs[obj].n;
            }
        }
        p.group_segs.push_back(segs);
        p.group_params.push_back(params);
    }
    if ((int)p.touched.size() > kMaxAdamSegs)
        return fail(c, PRENOM_ERR_INVALID_ARG, "a batched step updates at most %d objects", kMaxAdamSegs);
    if (!(op.flags & PRENOM_FLAG_NO_ADAM)) {
        AdamArgs &a = p.adam;
        a.beta1 = op.beta1;
        a.beta2 = op.beta2;
        a.eps = op.eps;
        a.n_segs = (int32_t)p.touched.size();
        a.chunk_start[0] = 0;
        for (size_t s = 0; s < p.touched.size(); ++s) {
            Object &o = c->objs[p.touched[s]];
            const int t = o.step + 1;
            const double c1 = 1.0 - pow((double)op.beta1, (double)t);
            const double c2 = 1.0 - pow((double)op.beta2, (double)t);
            p.adam_scal.push_back(make_float2((float)((double)op.lr / c1), (float)(1.0 / c2)));
            AdamSeg &sg = a.seg[s];
            sg.theta = o.theta;
            sg.grad = o.grad;
            sg.m = o.m;
            sg.v = o.v;
            sg.n = o.n;
            sg.skip = o.lss ? &o.lss->overflow : nullptr;
            sg.absmax = enc_absmax_ptr(o);
            sg.n_hash = o.n_hash;
            sg.mirror = o.feat16;
            a.chunk_start[s + 1] = a.chunk_start[s] + (o.n + kAdamChunk - 1) / kAdamChunk;
            if (o.lss && p.scales.n < kMaxScaleObjs)
                p.scales.s[p.scales.n++] = o.lss;
        }
        p.adam_grid = (int)std::min<int64_t>(a.chunk_start[a.n_segs], (int64_t)c->n_sm * 16);
    }
    return PRENOM_OK;
}

// Side streams and events for the concurrent groups of a batched step (created
// outside any graph capture).
cudaError_t ensure_side(prenom_ctx *c, size_t n_groups)
{
    const size_t n_side = n_groups > 1 ? n_groups - 1 : 0;
    int least = 0, greatest = 0;  // greatest is the numerically lowest
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    while (e == cudaSuccess && c->side.size() < n_side) {
        cudaStream_t s2 = nullptr;  // side stream i at the i-th greatest priority
        e = cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, std::min(greatest + (int)c->side.size(), least));
        if (e == cudaSuccess)
            c->side.push_back(s2);
    }
    while (e == cudaSuccess && c->side_ev.size() < n_side + 1) {
        cudaEvent_t ev2 = nullptr;
        e = cudaEventCreateWithFlags(&ev2, cudaEventDisableTiming);
        if (e == cudaSuccess)
            c->side_ev.push_back(ev2);
    }
    return e;
}

// Enqueues one batched step on the context's stream (also used under capture).
// group_ev (optional, groups + 1 events): recorded before each group's launches
// and after the last group's, so that group gi's device time lies between
// group_ev[gi] and group_ev[gi + 1].
// allow_fork: the groups may run concurrently: the group with the most
// parameters on the side stream of the greatest priority, the next on the next
// side stream, the one with the fewest on the context's stream; each forked
// group's Adam follows its kernels on its own stream, so that a group's Adam
// pass can start while other groups' kernels still run instead of waiting for
// the join.  *forked: whether it forked.
cudaError_t enqueue_batched(prenom_ctx *c, const Plan &p, const unsigned char *stage, size_t bytes, bool timed,
                            cudaEvent_t *group_ev = nullptr, bool allow_fork = false, bool *forked = nullptr)
{
    const size_t items_bytes = p.items.size() * sizeof(WorkItem);
    const WorkItem *d_items = reinterpret_cast<const WorkItem *>(c->d_work);
    const float2 *d_scal = reinterpret_cast<const float2 *>(c->d_work + items_bytes);
    cudaError_t e = cudaMemcpyAsync(c->d_work, stage, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = launch_zero_losses(d_items, (int)p.items.size(), c->stream);
    const WorkItem unused{};
    // groups run concurrently (their buffers are disjoint) where the step's tuning
    // chose it, never when kernels or groups are timed one by one; the side streams
    // exist already (ensure_side)
    const bool fork = allow_fork && !timed && !group_ev && c->stream != nullptr && p.groups.size() > 1 &&
                      c->side.size() + 1 >= p.groups.size() && c->side_ev.size() >= p.groups.size();
    const size_t n_side = fork ? p.groups.size() - 1 : 0;
    if (forked)
        *forked = fork;
    // stream slot of each group when forked: by parameter count, largest first
    std::vector<size_t> slot(p.groups.size());
    {
        std::vector<size_t> rank(p.groups.size());
        for (size_t gi = 0; gi < rank.size(); ++gi)
            rank[gi] = gi;
        std::stable_sort(rank.begin(), rank.end(),
                         [&](size_t a, size_t b) { return p.group_params[a] > p.group_params[b]; });
        for (size_t r = 0; r < rank.size(); ++r)
            slot[rank[r]] = r;
    }
    const bool group_adam = fork && p.adam_grid > 0;
    if (fork && e == cudaSuccess)
        e = cudaEventRecord(c->side_ev[0], c->stream);
    for (size_t i = 0; i < n_side && e == cudaSuccess; ++i)
        e = cudaStreamWaitEvent(c->side[i], c->side_ev[0], 0);
    for (size_t gi = 0; gi < p.groups.size(); ++gi) {
        const Group &g = p.groups[gi];
        cudaStream_t st = (fork && slot[gi] < n_side) ? c->side[slot[gi]] : c->stream;
        if (group_ev && e == cudaSuccess)
            e = cudaEventRecord(group_ev[gi], c->stream);
        if (e != cudaSuccess || g.total_tiles == 0)
            continue;
        const WorkList wl{d_items + g.first, g.count, g.total_tiles, g.hmax, g.split ? 1 : 0, g.feat16};
        cudaEvent_t ev;
        c->cur_group = timed ? group_index(c, group_label(g)) : -1;
        if (g.split) {
            if (timed)
                timed_begin(c, PRENOM_KERNEL_SAMPLE_ENCODE, &ev);
            e = launch_sample_encode(unused, wl, g.precision, g.enc_per_sm,
                                     grid_sample_encode(c, g.total_tiles, p.items[g.first].bd.rays_per_tile,
                                                        g.enc_per_sm),
                                     st);
            if (timed)
                timed_end(c, PRENOM_KERNEL_SAMPLE_ENCODE, ev);
            if (e != cudaSuccess)
                continue;
        }
        if (timed)
            timed_begin(c, PRENOM_KERNEL_TRAIN, &ev);
        e = g.precision == PRENOM_PRECISION_FP32 ? launch_fused_fp32_list(wl, g.W, g.IN, g.S, g.grid, st)
                                                 : launch_fused_tc_list(wl, g.W, g.IN, g.precision, g.grid, st);
        if (timed)
            timed_end(c, PRENOM_KERNEL_TRAIN, ev);
        if (g.split && e == cudaSuccess) {
            if (timed)
                timed_begin(c, PRENOM_KERNEL_SCATTER, &ev);
            e = launch_hash_scatter(unused, wl, grid_scatter(c, g.total_tiles), st, g.whole_runs);
            if (timed)
                timed_end(c, PRENOM_KERNEL_SCATTER, ev);
        }
    }
    // each forked group's Adam, on the group's stream after its kernels (also for a
    // group without tiles: its objects still take their step)
    for (size_t gi = 0; gi < p.groups.size() && group_adam && e == cudaSuccess; ++gi) {
        cudaStream_t st = slot[gi] < n_side ? c->side[slot[gi]] : c->stream;
        if (!p.group_segs[gi].empty()) {
            AdamArgs a{};
            a.beta1 = p.adam.beta1;
            a.beta2 = p.adam.beta2;
            a.eps = p.adam.eps;
            a.n_segs = (int32_t)p.group_segs[gi].size();
            a.chunk_start[0] = 0;
            for (int k = 0; k < a.n_segs; ++k) {
                const int sidx = p.group_segs[gi][k];
                a.seg[k] = p.adam.seg[sidx];
                a.seg[k].scal = d_scal + sidx;
                a.chunk_start[k + 1] = a.chunk_start[k] + (a.seg[k].n + kAdamChunk - 1) / kAdamChunk;
            }
            e = launch_adam(a, (int)std::min<int64_t>(a.chunk_start[a.n_segs], (int64_t)c->n_sm * 16), st);
        }
    }
    c->cur_group = -1;
    // the join (also after an error, so that a capture in progress ends with every stream joined)
    for (size_t i = 0; i < n_side && i + 1 < c->side_ev.size(); ++i) {
        cudaError_t e2 = cudaEventRecord(c->side_ev[1 + i], c->side[i]);
        if (e2 == cudaSuccess)
            e2 = cudaStreamWaitEvent(c->stream, c->side_ev[1 + i], 0);
        if (e == cudaSuccess)
            e = e2;
    }
    if (group_ev && e == cudaSuccess)
        e = cudaEventRecord(group_ev[p.groups.size()], c->stream);
    if (e == cudaSuccess && p.adam_grid > 0) {
        if (!group_adam) {
            AdamArgs a = p.adam;
            for (int s = 0; s < a.n_segs; ++s)
                a.seg[s].scal = d_scal + s;
            cudaEvent_t ev;
            if (timed)
                timed_begin(c, PRENOM_KERNEL_ADAM, &ev);
            e = launch_adam(a, p.adam_grid, c->stream);
            if (timed)
                timed_end(c, PRENOM_KERNEL_ADAM, ev);
        }
        if (e == cudaSuccess)
            e = launch_loss_scale_update_list(p.scales, c->stream);
    }
    return e;
}

int launches_of(const Plan &p, bool forked)
{
    int n = 1;  // loss reset
    for (const Group &g : p.groups)
        n += g.total_tiles > 0 ? (g.split ? 3 : 1) : 0;
    if (p.adam_grid > 0) {
        int adam = 1;
        if (forked) {  // one Adam per group with objects
            adam = 0;
            for (size_t gi = 0; gi < p.groups.size(); ++gi)
                adam += p.group_segs[gi].empty() ? 0 : 1;
        }
        n += adam + (p.scales.n > 0);
    }
    return n;
}

// capture_only: build the step's graph for the current staging buffer and keep
// it, without launching anything (the autotuner's set-up call).
int train_batched(prenom_ctx *c, const prenom_ray_batch *batches, int n, const prenom_train_opts &op, float *loss_dev,
                  bool capture_only = false)
{
    Plan p;
    int rc = plan_batched(c, batches, n, op, loss_dev, p);
    if (rc)
        return rc;
    // autotuner: the first calls of a group signature try each work-chunk size once
    bool tuning = false;
    const bool split_allowed = !(op.flags & PRENOM_FLAG_FUSED);
    const bool split_forced = split_allowed && (op.flags & PRENOM_FLAG_SPLIT);
    std::vector<std::string> gkeys;
    for (Group &g : p.groups) {
        gkeys.push_back(tune_key(g) + (split_allowed ? "/s" : "/f"));
        auto it = c->tune_best.find(gkeys.back());
        int cand;
        if (split_forced) {
            cand = 0;  // the split form, untuned
        } else if (it != c->tune_best.end()) {
            cand = it->second;
        } else {
            cand = (int)c->tune_ms[gkeys.back()].size() % tune_n(split_allowed);  // two rounds over the candidates
            tuning = true;
        }
        g.grid = group_grid(c, g, cand, split_allowed);
        g.split = cand_split(g, cand, split_allowed);
        g.whole_runs = cand_whole_runs(cand, split_allowed);
        g.enc_per_sm = cand_enc_per_sm(cand, split_allowed);
    }
    // once its groups are tuned, a step of several groups on a stream of its own
    // chooses between running them one after the other and concurrently on side
    // streams (forking fills the SMs one group's kernels leave idle, but the groups
    // then share L2): whole steps timed both ways, three rounds, the median counts
    std::string skey;
    int fork_trial = -1;  // this call times the step one after the other (0) or forked (1)
    bool allow_fork = false;
    if (!tuning && p.groups.size() > 1 && c->stream != nullptr && !c->timing) {
        for (const std::string &k : gkeys)
            skey += k + "|";
        auto fb = c->fork_best.find(skey);
        if (op.flags & PRENOM_FLAG_CONCURRENT)  // the caller's choice: no trial
            allow_fork = true;
        else if (fb != c->fork_best.end())
            allow_fork = fb->second;
        else
            fork_trial = (int)(c->fork_ms[skey].size() % 2);
    }
    // buffers of the split groups (planned before any staging or capture)
    size_t split_need = 0;
    for (const Group &g : p.groups)
        if (g.split)
            for (int j = g.first; j < g.first + g.count; ++j)
                split_need += split_bytes(p.items[j].bd.n_rays, p.items[j].bd.nr, p.items[j].bd.n_tiles);
    if (split_need) {
        if ((rc = ensure_split(c, split_need)))
            return rc;
        unsigned char *base = c->split_buf;
        for (const Group &g : p.groups)
            if (g.split)
                for (int j = g.first; j < g.first + g.count; ++j)
                    base += assign_split(p.items[j].bd, base);
    }
    // staging buffer: wait until the step that last read it has finished
    const size_t items_bytes = p.items.size() * sizeof(WorkItem);
    const size_t bytes = items_bytes + p.adam_scal.size() * sizeof(float2);
    const int b = c->stage_idx;
    cudaError_t e = cudaSuccess;
    if (c->stage_ev[b])
        e = cudaEventSynchronize(c->stage_ev[b]);
    if (e == cudaSuccess && bytes > c->h_stage_cap) {
        cudaStreamSynchronize(c->stream);
        for (int i = 0; i < 2; ++i) {
            cudaFreeHost(c->h_stage[i]);
            c->h_stage[i] = nullptr;
        }
        const size_t cap = std::max(bytes, (size_t)64 * sizeof(WorkItem));
        for (int i = 0; i < 2 && e == cudaSuccess; ++i)
            e = cudaMallocHost((void **)&c->h_stage[i], cap);
        c->h_stage_cap = e == cudaSuccess ? cap : 0;
        if (e == cudaSuccess) {
            cudaFree(c->d_work);
            c->d_work = nullptr;
            e = cudaMalloc(&c->d_work, cap);
            c->d_work_cap = e == cudaSuccess ? cap : 0;
        }
        for (auto &kv : c->graphs)  // captured graphs point at the old buffers
            cudaGraphExecDestroy(kv.second.exec);
        c->graphs.clear();
    }
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        if (!c->stage_ev[i])
            e = cudaEventCreateWithFlags(&c->stage_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess)
        return fail(c, e == cudaErrorMemoryAllocation ? PRENOM_ERR_OOM : PRENOM_ERR_CUDA, "batched step buffers: %s",
                    cudaGetErrorString(e));
    memcpy(c->h_stage[b], p.items.data(), items_bytes);
    if (!p.adam_scal.empty())
        memcpy(c->h_stage[b] + items_bytes, p.adam_scal.data(), p.adam_scal.size() * sizeof(float2));

    const bool use_graph = !tuning && fork_trial < 0 && !c->timing && c->stream != nullptr &&
                           !(op.flags & PRENOM_FLAG_NO_GRAPH);
    if (capture_only && !use_graph)
        return PRENOM_OK;  // nothing to capture (still tuning, timing on, legacy stream or graphs off)
    bool forked = false;  // the step's groups run concurrently (and each its own Adam)
    if (fork_trial >= 0) {
        c->n_tune_calls++;
        cudaEvent_t t0 = nullptr, t1 = nullptr;
        e = ensure_side(c, p.groups.size());
        if (e == cudaSuccess)
            e = cudaEventCreate(&t0);
        if (e == cudaSuccess)
            e = cudaEventCreate(&t1);
        if (e == cudaSuccess)
            e = cudaEventRecord(t0, c->stream);
        if (e == cudaSuccess)
            e = enqueue_batched(c, p, c->h_stage[b], bytes, false, nullptr, fork_trial == 1, &forked);
        if (e == cudaSuccess)
            e = cudaEventRecord(t1, c->stream);
        if (e == cudaSuccess)
            e = cudaEventSynchronize(t1);
        float ms = 0.f;
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, t0, t1);
        if (t0)
            cudaEventDestroy(t0);
        if (t1)
            cudaEventDestroy(t1);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "autotuner step");
        std::vector<float> &v = c->fork_ms[skey];
        v.push_back(ms);
        if ((int)v.size() == 2 * kTuneRounds) {
            float r[2][kTuneRounds];
            for (int q = 0; q < kTuneRounds; ++q)
                for (int f = 0; f < 2; ++f)
                    r[f][q] = v[(size_t)2 * q + f];
            std::sort(r[0], r[0] + kTuneRounds);
            std::sort(r[1], r[1] + kTuneRounds);
            c->fork_best[skey] = r[1][kTuneRounds / 2] < r[0][kTuneRounds / 2];
        }
    } else if (tuning) {
        c->n_tune_calls++;
        // each group is charged its own launches' device time, so that groups of one
        // step settle on candidates of their own
        std::vector<cudaEvent_t> gev(p.groups.size() + 1, nullptr);
        for (cudaEvent_t &x : gev)
            if (e == cudaSuccess)
                e = cudaEventCreate(&x);
        if (e == cudaSuccess)
            e = enqueue_batched(c, p, c->h_stage[b], bytes, false, gev.data());
        if (e == cudaSuccess)
            e = cudaEventSynchronize(gev.back());
        std::vector<float> gms(p.groups.size(), 0.f);
        for (size_t gi = 0; gi < p.groups.size() && e == cudaSuccess; ++gi)
            e = cudaEventElapsedTime(&gms[gi], gev[gi], gev[gi + 1]);
        for (cudaEvent_t x : gev)
            if (x)
                cudaEventDestroy(x);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "autotuner step");
        for (size_t gi = 0; gi < p.groups.size(); ++gi) {
            const float ms = gms[gi];
            std::vector<float> &v = c->tune_ms[gkeys[gi]];
            if (c->tune_best.count(gkeys[gi]) || split_forced)
                continue;
            if (!c->tune_warm.count(gkeys[gi])) {  // the first call loads modules and buffers: not timed
                c->tune_warm.insert(gkeys[gi]);
                continue;
            }
            v.push_back(ms);
            const int nc = tune_n(split_allowed);
            if ((int)v.size() == kTuneRounds * nc) {  // keep the candidate with the lowest median over its rounds
                int best = 0;
                float best_ms = INFINITY;
                for (int k = 0; k < nc; ++k) {
                    float r[kTuneRounds];
                    for (int q = 0; q < kTuneRounds; ++q)
                        r[q] = v[(size_t)q * nc + k];
                    std::sort(r, r + kTuneRounds);
                    if (r[kTuneRounds / 2] < best_ms) {
                        best_ms = r[kTuneRounds / 2];
                        best = k;
                    }
                }
                c->tune_best[gkeys[gi]] = best;
            }
        }
    } else if (use_graph) {
        std::string key = std::to_string(b) + ":" + std::to_string(bytes) + ":" + std::to_string(p.adam_grid);
        key += allow_fork ? "F" : "S";
        for (const Group &g : p.groups)
            key += "|" + group_key(g) + "/" + std::to_string(g.grid) + (g.split ? (g.whole_runs ? "w" : "s") : "f") +
                   std::to_string(g.enc_per_sm);
        for (int32_t id : p.touched)
            key += "," + std::to_string(id);
        char tail[96];
        snprintf(tail, sizeof(tail), "#%a/%a/%a", (double)op.beta1, (double)op.beta2, (double)op.eps);
        key += tail;
        auto it = c->graphs.find(key);
        if (it == c->graphs.end()) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            e = ensure_side(c, p.groups.size());
            if (e == cudaSuccess)
                e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const cudaError_t e1 = enqueue_batched(c, p, c->h_stage[b], bytes, false, nullptr, allow_fork, &forked);
                e = cudaStreamEndCapture(c->stream, &graph);
                if (e == cudaSuccess)
                    e = e1;
            }
            if (e == cudaSuccess)  // the forked groups keep their side streams' priorities
                e = cudaGraphInstantiateWithFlags(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
            if (graph)
                cudaGraphDestroy(graph);
            if (e != cudaSuccess)
                return cuda_fail(c, e, "batched step graph capture");
            c->n_captures++;
            if (c->graphs.size() >= kMaxGraphs) {  // evict the least recently used signature
                auto old = c->graphs.begin();
                for (auto g = c->graphs.begin(); g != c->graphs.end(); ++g)
                    if (g->second.last_use < old->second.last_use)
                        old = g;
                cudaStreamSynchronize(c->stream);  // it may still be running
                cudaGraphExecDestroy(old->second.exec);
                c->graphs.erase(old);
            }
            it = c->graphs.emplace(key, prenom_ctx::CachedGraph{exec, 0}).first;
        }
        it->second.last_use = ++c->graph_tick;
        forked = allow_fork && p.groups.size() > 1;  // as when the graph was captured (side streams made first)
        if (capture_only) {  // kept for the step that will use this staging buffer
            c->stage_idx ^= 1;
            return PRENOM_OK;
        }
        e = cudaGraphLaunch(it->second.exec, c->stream);
    } else {
        const int64_t before = c->launches;  // timed launches count themselves; the total is set below
        e = c->timing ? cudaSuccess : ensure_side(c, p.groups.size());
        if (e == cudaSuccess)
            e = enqueue_batched(c, p, c->h_stage[b], bytes, c->timing, nullptr, allow_fork, &forked);
        c->launches = before;
    }
    if (e == cudaSuccess)
        e = cudaEventRecord(c->stage_ev[b], c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "batched step");
    c->stage_idx ^= 1;
    c->launches += launches_of(p, forked);
    if (!(op.flags & PRENOM_FLAG_NO_ADAM))
        for (int32_t id : p.touched)
            c->objs[id].step += 1;
    return PRENOM_OK;
}

// Whether some group signature of this step still has autotuner calls ahead.
bool tuning_pending(prenom_ctx *c, const prenom_ray_batch *batches, int n, const prenom_train_opts &op, int *rc)
{
    Plan p;
    *rc = plan_batched(c, batches, n, op, nullptr, p);
    if (*rc)
        return false;
    const bool split_allowed = !(op.flags & PRENOM_FLAG_FUSED);
    const bool split_forced = split_allowed && (op.flags & PRENOM_FLAG_SPLIT);  // groups untuned
    std::string skey;
    for (const Group &g : p.groups) {
        const std::string k = tune_key(g) + (split_allowed ? "/s" : "/f");
        if (!split_forced && !c->tune_best.count(k))
            return true;
        skey += k + "|";
    }
    return p.groups.size() > 1 && c->stream != nullptr && !c->timing && !(op.flags & PRENOM_FLAG_CONCURRENT) &&
           !c->fork_best.count(skey);
}

}  // namespace

namespace prenom {

// Field descriptor for parameters held in caller-owned buffers (used by the
// allocation-free training step).  Validates the architecture with the same
// rules as prenom_create_object; failures set the context-free last error.
int describe_caller_field(const prenom_arch *arch, const float *theta, float *grad, const float *grid, int32_t R,
                          ObjDesc *od, int64_t *n_params)
{
    const int rc = check_arch(nullptr, arch);
    if (rc)
        return rc;
    Object o;
    o.arch = *arch;
    level_geometry(*arch, o);
    o.theta = const_cast<float *>(theta);
    o.grid = const_cast<float *>(grid);
    o.R = R;
    *od = make_objdesc(o, grad);
    *n_params = o.n;
    return PRENOM_OK;
}

// The step options checked as prenom_train_step checks them (Adam constants
// included); failures set the context-free last error.
int check_caller_opts(const prenom_train_opts *op)
{
    return check_opts(nullptr, op, true);
}

int set_context_free_error(int code, const char *msg)
{
    return fail(nullptr, code, "%s", msg);
}

}  // namespace prenom

extern "C" {

int prenom_create(prenom_ctx **out, void *cuda_stream, uint64_t seed)
{
    if (!out)
        return fail(nullptr, PRENOM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    prenom_ctx *c = new (std::nothrow) prenom_ctx();
    if (!c)
        return fail(nullptr, PRENOM_ERR_OOM, "host allocation failed");
    c->stream = (cudaStream_t)cuda_stream;
    c->seed = seed;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device);
    int optin = 0;
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    if (e == cudaSuccess) {
        int major = 0;
        e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, c->device);
        if (e == cudaSuccess && major < 10) {
            delete c;
            return fail(nullptr, PRENOM_ERR_CUDA, "device compute capability %d.x: this library is built for sm_103a",
                        major);
        }
    }
    if (e == cudaSuccess)
        e = cudaMalloc(&c->scratch, kScratchLosses * sizeof(float));
    if (e == cudaSuccess)
        e = cudaMalloc(&c->status, 4 * sizeof(int32_t));
    if (e == cudaSuccess)
        e = cudaMemset(c->status, 0, 4 * sizeof(int32_t));
    if (e != cudaSuccess) {
        const int code = (e == cudaErrorMemoryAllocation) ? PRENOM_ERR_OOM : PRENOM_ERR_CUDA;
        fail(nullptr, code, "context creation: %s", cudaGetErrorString(e));
        delete c;
        return code;
    }
    c->smem_optin = (size_t)optin;
    *out = c;
    return PRENOM_OK;
}

void prenom_destroy(prenom_ctx *c)
{
    if (!c)
        return;
    cudaStreamSynchronize(c->stream);
    for (auto &o : c->objs) {
        cudaFree(o.arena);
        cudaFree(o.grid);
        cudaFree(o.lss);
    }
    cudaFree(c->status);
    for (auto &kv : c->graphs)
        cudaGraphExecDestroy(kv.second.exec);
    for (int i = 0; i < 2; ++i) {
        cudaFreeHost(c->h_stage[i]);
        if (c->stage_ev[i])
            cudaEventDestroy(c->stage_ev[i]);
    }
    for (cudaStream_t s2 : c->side)
        cudaStreamDestroy(s2);
    for (cudaEvent_t ev2 : c->side_ev)
        cudaEventDestroy(ev2);
    cudaFree(c->d_work);
    cudaFree(c->split_buf);
    cudaFree(c->query_buf);
    cudaFree(c->rays_buf);
    for (auto &p : c->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->ev_free)
        cudaEventDestroy(e);
    cudaFree(c->scratch);
    delete c;
}

const char *prenom_last_error(const prenom_ctx *c)
{
    return c ? c->err.c_str() : g_create_error.c_str();
}

int prenom_create_object(prenom_ctx *c, const prenom_arch *arch, const float *init_params, int32_t *obj_out)
{
    if (!c)
        return fail(nullptr, PRENOM_ERR_INVALID_ARG, "ctx is NULL");
    if (!obj_out)
        return fail(c, PRENOM_ERR_INVALID_ARG, "obj_out is NULL");
    int rc = check_arch(c, arch);
    if (rc)
        return rc;
    Object o;
    o.arch = *arch;
    level_geometry(*arch, o);
    // theta | grad | m | v, each n_pad floats, then (BF16 features) the tables' copy
    const int64_t mirror_floats = arch->features == PRENOM_FEATURES_BF16 ? (o.n_hash / 2 + 63) / 64 * 64 : 0;
    const int64_t arena_floats = o.n_pad * 4 + mirror_floats;
    cudaError_t e = cudaMalloc(&o.arena, (size_t)arena_floats * sizeof(float));
    if (e != cudaSuccess)
        return fail(c, PRENOM_ERR_OOM, "object arena of %lld floats: %s", (long long)arena_floats,
                    cudaGetErrorString(e));
    o.theta = o.arena;
    o.grad = o.arena + o.n_pad;
    o.m = o.arena + 2 * o.n_pad;
    o.v = o.arena + 3 * o.n_pad;
    o.feat16 = mirror_floats ? reinterpret_cast<uint16_t *>(o.arena + 4 * o.n_pad) : nullptr;
    e = cudaMemsetAsync(o.grad, 0, (size_t)o.n_pad * 3 * sizeof(float), c->stream);
    if (e == cudaSuccess) {
        if (init_params) {
            e = cudaMemcpyAsync(o.theta, init_params, (size_t)o.n * sizeof(float), cudaMemcpyDefault, c->stream);
        } else {
            int32_t shape[8];
            const int nl = arch->hidden + 1;
            for (int l = 0; l < nl; ++l) {
                shape[2 * l] = (l == arch->hidden) ? 4 : arch->width;
                shape[2 * l + 1] = (l == 0) ? o.IN : arch->width;
            }
            cudaEvent_t ev;
            timed_begin(c, PRENOM_KERNEL_INIT, &ev);
            e = launch_init_params(o.theta, o.n_hash, shape, nl, c->seed, (uint32_t)c->objs.size(), c->n_sm * 4,
                                   c->stream);
            timed_end(c, PRENOM_KERNEL_INIT, ev);
        }
    }
    if (e == cudaSuccess && arch->precision != PRENOM_PRECISION_FP32) {
        e = cudaMalloc(&o.lss, sizeof(LossScaleState));
        if (e == cudaSuccess) {
            const bool fp16 = arch->precision == PRENOM_PRECISION_FP16;
            const LossScaleState init{fp16 ? 32768.f : 1.f, 0, 0, 0, kLossScaleGrowth, fp16 ? 1 : 0, 1.f, 0u,
                                      o.theta + o.n_hash, o.IN, arch->width, arch->hidden};
            e = cudaMemcpyAsync(o.lss, &init, sizeof(init), cudaMemcpyHostToDevice, c->stream);
        }
    }
    if (e == cudaSuccess && refresh_enc_scale(c, o) != PRENOM_OK)
        e = cudaErrorLaunchFailure;
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaFree(o.arena);
        cudaFree(o.lss);
        return cuda_fail(c, e, "object initialisation");
    }
    o.alive = true;
    c->objs.push_back(o);
    *obj_out = (int32_t)(c->objs.size() - 1);
    return PRENOM_OK;
}

int prenom_destroy_object(prenom_ctx *c, int32_t obj)
{
    Object *o = get_obj(c, obj);
    if (!o)
        return fail(c, PRENOM_ERR_INVALID_ARG, "unknown object %d", obj);
    cudaStreamSynchronize(c->stream);
    cudaFree(o->arena);
    cudaFree(o->grid);
    cudaFree(o->lss);
    *o = Object();
    return PRENOM_OK;
}

int prenom_param_count(prenom_ctx *c, int32_t obj, size_t *n)
{
    Object *o = get_obj(c, obj);
    if (!o || !n)
        return fail(c, PRENOM_ERR_INVALID_ARG, "unknown object %d or NULL output", obj);
    *n = (size_t)o->n;
    return PRENOM_OK;
}

int prenom_arch_param_count(const prenom_arch *arch, size_t *n)
{
    if (!arch || !n)
        return fail(nullptr, PRENOM_ERR_INVALID_ARG, "arch and n are required");
    const int rc = check_arch(nullptr, arch);
    if (rc)
        return rc;
    Object o;
    o.arch = *arch;
    level_geometry(*arch, o);
    *n = (size_t)o.n;
    return PRENOM_OK;
}

int prenom_level_info(prenom_ctx *c, int32_t obj, int32_t *res, int64_t *offset, int32_t *dense)
{
    Object *o = get_obj(c, obj);
    if (!o)
        return fail(c, PRENOM_ERR_INVALID_ARG, "unknown object %d", obj);
    for (int l = 0; l < o->arch.L; ++l) {
        if (res)
            res[l] = o->res[l];
        if (dense)
            dense[l] = o->dense[l];
    }
    if (offset)
        for (int l = 0; l <= o->arch.L; ++l)
            offset[l] = o->off[l];
    return PRENOM_OK;
}

int prenom_set_prior_grid(prenom_ctx *c, int32_t obj, const float *grid, int32_t res)
{
    Object *o = get_obj(c, obj);
    if (!o)
        return fail(c, PRENOM_ERR_INVALID_ARG, "unknown object %d", obj);
    if (!grid || res < 2 || res > 1024)
        return fail(c, PRENOM_ERR_INVALID_ARG, "grid must be non-NULL with 2 <= res <= 1024");
    const size_t bytes = (size_t)res * res * res * sizeof(float);
    if (o->R != res) {
        cudaStreamSynchronize(c->stream);
        cudaFree(o->grid);
        o->grid = nullptr;
        o->R = 0;
        const cudaError_t e = cudaMalloc(&o->grid, bytes);
        if (e != cudaSuccess)
            return fail(c, PRENOM_ERR_OOM, "prior grid %d^3: %s", res, cudaGetErrorString(e));
        o->R = res;
    }
    const cudaError_t e = cudaMemcpyAsync(o->grid, grid, bytes, cudaMemcpyDefault, c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "prior grid copy");
    return PRENOM_OK;
}

int prenom_train_step(prenom_ctx *c, const prenom_ray_batch *batches, int32_t n_batches,
                      const prenom_train_opts *op, float *loss_dev)
{
    if (!c)
        return fail(nullptr, PRENOM_ERR_INVALID_ARG, "ctx is NULL");
    if (n_batches < 0 || (n_batches > 0 && !batches))
        return fail(c, PRENOM_ERR_INVALID_ARG, "bad batch list");
    int rc = check_opts(c, op, true);
    if (rc)
        return rc;
    for (int i = 0; i < n_batches; ++i)
        if ((rc = check_batch(c, batches[i], true)))
            return rc;
    for (int i = 0; i < n_batches; ++i) {
        Object &o = c->objs[batches[i].obj];
        if (o.lss && o.step == 0 && op->loss_scale_init > 0.f) {  // caller-chosen starting scale
            const float s0 = op->loss_scale_init;
            const cudaError_t e = cudaMemcpyAsync(&o.lss->scale, &s0, sizeof(float), cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess)
                cudaStreamSynchronize(c->stream);
        }
    }
    if (n_batches > 0 && !(op->flags & PRENOM_FLAG_CHECK_FINITE))
        return train_batched(c, batches, n_batches, *op, loss_dev);
    // the finiteness check reads every batch's loss: without loss_dev they go to
    // the context's scratch slots
    const bool check = (op->flags & PRENOM_FLAG_CHECK_FINITE) && n_batches > 0;
    if (check && !loss_dev) {
        if (n_batches > kScratchLosses)
            return fail(c, PRENOM_ERR_INVALID_ARG, "PRENOM_FLAG_CHECK_FINITE with more than %d batches needs loss_dev",
                        kScratchLosses);
        loss_dev = c->scratch;
    }
    if (loss_dev && n_batches > 0) {
        const cudaError_t e = cudaMemsetAsync(loss_dev, 0, (size_t)n_batches * sizeof(float), c->stream);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "loss reset");
    }
    std::vector<int32_t> touched;
    for (int i = 0; i < n_batches; ++i) {
        const prenom_ray_batch &b = batches[i];
        Object &o = c->objs[b.obj];
        ObjDesc od = make_objdesc(o, o.grad);
        BatchDesc bd = make_batchdesc(c, o, b, *op, kTrain, 128);
        bd.loss = loss_dev ? loss_dev + i : c->scratch;
        if ((rc = launch_fused(c, o, od, bd, PRENOM_KERNEL_TRAIN, !(op->flags & PRENOM_FLAG_FUSED))))
            return rc;
        if (std::find(touched.begin(), touched.end(), b.obj) == touched.end())
            touched.push_back(b.obj);
    }
    if (check) {
        std::vector<float> h(n_batches);
        const cudaError_t e = cudaMemcpyAsync(h.data(), loss_dev, h.size() * sizeof(float), cudaMemcpyDeviceToHost,
                                              c->stream);
        if (e == cudaSuccess)
            cudaStreamSynchronize(c->stream);
        for (float v : h)
            if (!isfinite(v)) {
                for (int32_t id : touched)
                    cudaMemsetAsync(c->objs[id].grad, 0, (size_t)c->objs[id].n * sizeof(float), c->stream);
                return fail(c, PRENOM_ERR_NONFINITE, "non-finite loss; gradients dropped, no Adam step");
            }
    }
    if (op->flags & PRENOM_FLAG_NO_ADAM)
        return PRENOM_OK;
    return run_adam(c, touched, *op);
}

int prenom_autotune(prenom_ctx *c, const prenom_ray_batch *batches, int32_t n_batches, const prenom_train_opts *op)
{
    if (!c)
        return fail(nullptr, PRENOM_ERR_INVALID_ARG, "ctx is NULL");
    if (n_batches < 0 || (n_batches > 0 && !batches))
        return fail(c, PRENOM_ERR_INVALID_ARG, "bad batch list");
    int rc = check_opts(c, op, true);
    if (rc)
        return rc;
    for (int i = 0; i < n_batches; ++i)
        if ((rc = check_batch(c, batches[i], true)))
            return rc;
    if (n_batches == 0 || (op->flags & PRENOM_FLAG_CHECK_FINITE))
        return PRENOM_OK;  // such steps are neither tuned nor captured
    if (op->flags & PRENOM_FLAG_RETUNE) {  // forget the step's groups' and its step-level choices
        Plan p;
        if ((rc = plan_batched(c, batches, n_batches, *op, nullptr, p)))
            return rc;
        const bool split_allowed = !(op->flags & PRENOM_FLAG_FUSED);
        std::string skey;
        for (const Group &g : p.groups) {
            const std::string k = tune_key(g) + (split_allowed ? "/s" : "/f");
            c->tune_best.erase(k);
            c->tune_ms.erase(k);
            skey += k + "|";
        }
        c->fork_best.erase(skey);
        c->fork_ms.erase(skey);
    }
    // the autotuner's calls, as gradient-only steps (no Adam, no step count)
    prenom_train_opts t = *op;
    t.flags |= PRENOM_FLAG_NO_ADAM;
    t.flags &= ~PRENOM_FLAG_RETUNE;
    for (int i = 0; i < 2 + (kTuneNSplit + 2) * kTuneRounds; ++i) {
        const bool pending = tuning_pending(c, batches, n_batches, t, &rc);
        if (rc)
            return rc;
        if (!pending)
            break;
        if ((rc = train_batched(c, batches, n_batches, t, nullptr)))
            return rc;
    }
    // undo what those calls left behind: accumulated gradients, overflow flags
    std::set<int32_t> seen;
    for (int i = 0; i < n_batches; ++i) {
        Object &o = c->objs[batches[i].obj];
        if (!seen.insert(batches[i].obj).second)
            continue;
        cudaError_t e = cudaMemsetAsync(o.grad, 0, (size_t)o.n * sizeof(float), c->stream);
        if (e == cudaSuccess && o.lss)
            e = cudaMemsetAsync(&o.lss->overflow, 0, sizeof(int32_t), c->stream);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "autotune clean-up");
    }
    // the step's graphs, one per staging buffer, captured now and launched by later steps
    for (int i = 0; i < 2; ++i)
        if ((rc = train_batched(c, batches, n_batches, *op, nullptr, true)))
            return rc;
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? PRENOM_OK : cuda_fail(c, e, "autotune");
}

int prenom_render(prenom_ctx *c, const prenom_ray_batch *b, const prenom_train_opts *op, float *rgb, float *depth,
                  float *acc, int32_t *bins_out, float *t_out)
{
    if (!c)
        return fail(nullptr, PRENOM_ERR_INVALID_ARG, "ctx is NULL");
    if (!b)
        return fail(c, PRENOM_ERR_INVALID_ARG, "batch is NULL");
    int rc = check_opts(c, op, false);
    if (rc || (rc = check_batch(c, *b, false)))
        return rc;
    Object &o = c->objs[b->obj];
    ObjDesc od = make_objdesc(o, nullptr);
    BatchDesc bd = make_batchdesc(c, o, *b, *op, kRender, 128);
    bd.out_rgb = rgb;
    bd.out_depth = depth;
    bd.out_acc = acc;
    bd.out_bins = bins_out;
    bd.out_t = t_out;
    bd.loss = c->scratch;
    return launch_fused(c, o, od, bd, PRENOM_KERNEL_RENDER);
}

int prenom_render_backward(prenom_ctx *c, const prenom_ray_batch *b, const prenom_train_opts *op, const float *d_out,
                           float *grad)
{
    if (!c)
        return fail(nullptr, PRENOM_ERR_INVALID_ARG, "ctx is NULL");
    if (!b || !grad || (b->n_rays > 0 && !d_out))
        return fail(c, PRENOM_ERR_INVALID_ARG, "batch, d_out and grad are required");
    if (reinterpret_cast<uintptr_t>(grad) % 16 != 0)
        return fail(c, PRENOM_ERR_INVALID_ARG, "grad is not 16-byte aligned");
    int rc = check_opts(c, op, false);
    if (rc || (rc = check_batch(c, *b, false)))
        return rc;
    Object &o = c->objs[b->obj];
    ObjDesc od = make_objdesc(o, grad);
    BatchDesc bd = make_batchdesc(c, o, *b, *op, kRenderBwd, 128);
    bd.upstream = d_out;
    bd.loss = c->scratch;
    return launch_fused(c, o, od, bd, PRENOM_KERNEL_RENDER_BWD);
}

static float *state_ptr(Object *o, int32_t which)
{
    switch (which) {
    case PRENOM_STATE_THETA: return o->theta;
    case PRENOM_STATE_GRAD: return o->grad;
    case PRENOM_STATE_ADAM_M: return o->m;
    case PRENOM_STATE_ADAM_V: return o->v;
    default: return nullptr;
    }
}

int prenom_get_state(prenom_ctx *c, int32_t obj, int32_t which, float *dst, size_t n)
{
    Object *o = get_obj(c, obj);
    if (!o || !dst || (size_t)o->n != n || !state_ptr(o, which))
        return fail(c, PRENOM_ERR_INVALID_ARG, "get_state: bad object, buffer, size or selector");
    cudaError_t e = cudaMemcpyAsync(dst, state_ptr(o, which), n * sizeof(float), cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? PRENOM_OK : cuda_fail(c, e, "get_state");
}

int prenom_set_state(prenom_ctx *c, int32_t obj, int32_t which, const float *src, size_t n)
{
    Object *o = get_obj(c, obj);
    if (!o || !src || (size_t)o->n != n || !state_ptr(o, which))
        return fail(c, PRENOM_ERR_INVALID_ARG, "set_state: bad object, buffer, size or selector");
    cudaError_t e = cudaMemcpyAsync(state_ptr(o, which), src, n * sizeof(float), cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && which == PRENOM_STATE_THETA && refresh_enc_scale(c, *o) != PRENOM_OK)
        return PRENOM_ERR_CUDA;
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? PRENOM_OK : cuda_fail(c, e, "set_state");
}

int prenom_get_step(prenom_ctx *c, int32_t obj, int32_t *step)
{
    Object *o = get_obj(c, obj);
    if (!o || !step)
        return fail(c, PRENOM_ERR_INVALID_ARG, "unknown object %d or NULL output", obj);
    *step = o->step;
    return PRENOM_OK;
}

int prenom_set_step(prenom_ctx *c, int32_t obj, int32_t step)
{
    Object *o = get_obj(c, obj);
    if (!o || step < 0)
        return fail(c, PRENOM_ERR_INVALID_ARG, "unknown object %d or negative step", obj);
    o->step = step;
    return PRENOM_OK;
}

// ------------------------------------------------------------- Reptile
static bool same_layout(const prenom_arch &a, const prenom_arch &b)
{
    return a.L == b.L && a.F == b.F && a.log2T == b.log2T && a.n_min == b.n_min && a.n_max == b.n_max &&
           a.width == b.width && a.hidden == b.hidden;
}

// Validates a meta object and its tasks and fills the task pointers of a.
static int reptile_args(prenom_ctx *c, int32_t meta, const int32_t *tasks, int32_t n_tasks, ReptileArgs &a,
                        Object **meta_out)
{
    if (!c)
        return fail(nullptr, PRENOM_ERR_INVALID_ARG, "ctx is NULL");
    if (n_tasks < 1 || n_tasks > kMaxReptileTasks || !tasks)
        return fail(c, PRENOM_ERR_INVALID_ARG, "1..%d task objects are required", kMaxReptileTasks);
    Object *m = meta >= 0 ? get_obj(c, meta) : nullptr;
    if (meta >= 0 && !m)
        return fail(c, PRENOM_ERR_INVALID_ARG, "unknown meta object %d", meta);
    const Object *first = nullptr;
    for (int i = 0; i < n_tasks; ++i) {
        Object *t = get_obj(c, tasks[i]);
        if (!t)
            return fail(c, PRENOM_ERR_INVALID_ARG, "unknown task object %d", tasks[i]);
        if (tasks[i] == meta)
            return fail(c, PRENOM_ERR_INVALID_ARG, "the meta object cannot be one of its tasks");
        for (int j = 0; j < i; ++j)
            if (tasks[j] == tasks[i])
                return fail(c, PRENOM_ERR_INVALID_ARG, "task object %d is listed twice", tasks[i]);
        const Object *ref = m ? m : (first ? first : t);
        if (!same_layout(t->arch, ref->arch))
            return fail(c, PRENOM_ERR_INVALID_ARG, "task object %d has another architecture", tasks[i]);
        first = first ? first : t;
        a.theta[i] = t->theta;
    }
    a.n_tasks = n_tasks;
    a.n = first->n;
    a.n_pad = first->n_pad;
    if (meta_out)
        *meta_out = m;
    return PRENOM_OK;
}

static int reptile_launch(prenom_ctx *c, const ReptileArgs &a, int op)
{
    const int64_t work = (a.n + 3) / 4;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)c->n_sm * 8));
    const cudaError_t e = launch_reptile(a, op, grid, c->stream);
    c->launches++;
    return e == cudaSuccess ? PRENOM_OK : cuda_fail(c, e, "Reptile kernel launch");
}

int prenom_reptile_begin(prenom_ctx *c, int32_t meta, const int32_t *tasks, int32_t n_tasks)
{
    ReptileArgs a{};
    Object *m = nullptr;
    int rc = meta < 0 ? fail(c, PRENOM_ERR_INVALID_ARG, "a meta object is required")
                      : reptile_args(c, meta, tasks, n_tasks, a, &m);
    if (rc)
        return rc;
    a.meta = m->theta;
    if ((rc = reptile_launch(c, a, kReptileBroadcast)))
        return rc;
    for (int i = 0; i < n_tasks; ++i) {
        c->objs[tasks[i]].step = 0;
        if ((rc = refresh_enc_scale(c, c->objs[tasks[i]])))
            return rc;
    }
    return PRENOM_OK;
}

int prenom_reptile_update(prenom_ctx *c, int32_t meta, const int32_t *tasks, int32_t n_tasks, float beta)
{
    ReptileArgs a{};
    Object *m = nullptr;
    int rc = meta < 0 ? fail(c, PRENOM_ERR_INVALID_ARG, "a meta object is required")
                      : reptile_args(c, meta, tasks, n_tasks, a, &m);
    if (rc)
        return rc;
    if (!(beta >= 0.f && beta <= 1.f))
        return fail(c, PRENOM_ERR_INVALID_ARG, "beta must lie in [0, 1]");
    a.meta = m->theta;
    a.beta = beta;
    a.nf = (float)n_tasks;
    if ((rc = reptile_launch(c, a, kReptileSum)))
        return rc;
    return refresh_enc_scale(c, *m);
}

int prenom_reptile_task_sum(prenom_ctx *c, const int32_t *tasks, int32_t n_tasks, float *sum)
{
    ReptileArgs a{};
    int rc = reptile_args(c, -1, tasks, n_tasks, a, nullptr);
    if (rc)
        return rc;
    if (!sum || reinterpret_cast<uintptr_t>(sum) % 16 != 0)
        return fail(c, PRENOM_ERR_INVALID_ARG, "sum must be a 16-byte aligned device buffer");
    a.sum = sum;
    return reptile_launch(c, a, kReptileSum);
}

int prenom_reptile_apply(prenom_ctx *c, int32_t meta, const float *sum, int32_t n_total, float beta)
{
    if (!c)
        return fail(nullptr, PRENOM_ERR_INVALID_ARG, "ctx is NULL");
    Object *m = get_obj(c, meta);
    if (!m)
        return fail(c, PRENOM_ERR_INVALID_ARG, "unknown meta object %d", meta);
    if (!sum || reinterpret_cast<uintptr_t>(sum) % 16 != 0)
        return fail(c, PRENOM_ERR_INVALID_ARG, "sum must be a 16-byte aligned device buffer");
    if (n_total < 1 || !(beta >= 0.f && beta <= 1.f))
        return fail(c, PRENOM_ERR_INVALID_ARG, "n_total >= 1 and beta in [0, 1] are required");
    ReptileArgs a{};
    a.n = m->n;
    a.n_pad = m->n_pad;
    a.meta = m->theta;
    a.sum = const_cast<float *>(sum);
    a.beta = beta;
    a.nf = (float)n_total;
    const int rc = reptile_launch(c, a, kReptileApply);
    return rc ? rc : refresh_enc_scale(c, *m);
}

// ------------------------------------------------- prior grid and Eq. 3
static int ensure_query(prenom_ctx *c, size_t bytes)
{
    if (bytes <= c->query_cap)
        return PRENOM_OK;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "stream");
    cudaFree(c->query_buf);
    cudaFree(c->rays_buf);
    c->query_buf = nullptr;
    c->query_cap = 0;
    e = cudaMalloc(&c->query_buf, bytes);
    if (e != cudaSuccess)
        return fail(c, PRENOM_ERR_OOM, "query buffers of %zu bytes: %s", bytes, cudaGetErrorString(e));
    c->query_cap = bytes;
    return PRENOM_OK;
}

int prenom_make_rays(prenom_ctx *c, const prenom_keyframe *kfs, int32_t n_kf, const prenom_object_state *st,
                     int32_t n_rays, const uint32_t *draws, float *o, float *d, float *rgb, float *depth,
                     uint8_t *is_obj, int64_t *n_candidates)
{
    if (!c)
        return fail(nullptr, PRENOM_ERR_INVALID_ARG, "ctx is NULL");
    if (!kfs || n_kf < 1 || n_kf > 4096 || !st || n_rays < 0)
        return fail(c, PRENOM_ERR_INVALID_ARG, "1..4096 keyframes, an object state and n_rays >= 0 are required");
    if (n_rays > 0 && (!o || !d || !rgb || !depth || !is_obj))
        return fail(c, PRENOM_ERR_INVALID_ARG, "o, d, rgb, depth and is_obj are required");
    for (int a = 0; a < 3; ++a)
        if (!(st->size[a] > 0.f) || !isfinite(st->size[a]))
            return fail(c, PRENOM_ERR_INVALID_ARG, "object size must be finite and > 0");
    std::vector<int64_t> off(n_kf + 1, 0);
    for (int k = 0; k < n_kf; ++k) {
        const prenom_keyframe &f = kfs[k];
        if (f.width < 1 || f.height < 1 || !f.rgb || !f.depth || !f.mask || !(f.fx != 0.f) || !(f.fy != 0.f))
            return fail(c, PRENOM_ERR_INVALID_ARG, "keyframe %d: size, images and intrinsics are required", k);
        off[k + 1] = off[k] + (int64_t)f.width * f.height;
    }
    const int64_t n_pix = off[n_kf];
    if (n_pix >= ((int64_t)1 << 31))
        return fail(c, PRENOM_ERR_INVALID_ARG, "at most 2^31 - 1 pixels per call");
    const size_t kf_bytes = ((size_t)n_kf * sizeof(prenom_keyframe) + 255) / 256 * 256;
    const size_t off_bytes = ((size_t)(n_kf + 1) * sizeof(int64_t) + 255) / 256 * 256;
    const size_t need = kf_bytes + off_bytes + make_rays_scratch(n_pix);
    if (need > c->rays_cap) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "stream");
        cudaFree(c->rays_buf);
        c->rays_buf = nullptr;
        c->rays_cap = 0;
        e = cudaMalloc(&c->rays_buf, need);
        if (e != cudaSuccess)
            return fail(c, PRENOM_ERR_OOM, "ray-generation buffers of %zu bytes: %s", need, cudaGetErrorString(e));
        c->rays_cap = need;
    }
    prenom_keyframe *d_kf = reinterpret_cast<prenom_keyframe *>(c->rays_buf);
    int64_t *d_off = reinterpret_cast<int64_t *>(c->rays_buf + kf_bytes);
    cudaError_t e = cudaMemcpyAsync(d_kf, kfs, (size_t)n_kf * sizeof(prenom_keyframe), cudaMemcpyHostToDevice,
                                    c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream);
    int64_t *d_count = nullptr;
    if (e == cudaSuccess)
        e = launch_make_rays(d_kf, d_off, n_kf, n_pix, *st, c->rays_buf + kf_bytes + off_bytes, n_rays, draws,
                             c->seed, c->ray_calls, o, d, rgb, depth, is_obj, &d_count, c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "ray generation");
    c->ray_calls += 1;
    c->launches += n_pix > 0 ? 3 + (n_rays > 0) : (n_rays > 0);
    if (n_candidates) {
        e = cudaMemcpyAsync(n_candidates, d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "candidate count");
    }
    return PRENOM_OK;
}

int prenom_density_grid(prenom_ctx *c, int32_t obj, int32_t res, float *grid_out)
{
    if (!c)
        return fail(nullptr, PRENOM_ERR_INVALID_ARG, "ctx is NULL");
    Object *o = get_obj(c, obj);
    if (!o)
        return fail(c, PRENOM_ERR_INVALID_ARG, "unknown object %d", obj);
    if (!grid_out || res < kMinNr || res > 64)
        return fail(c, PRENOM_ERR_INVALID_ARG, "grid_out must be non-NULL with %d <= res <= 64", kMinNr);
    const size_t rays = (size_t)res * res, pts = rays * res;
    int rc = ensure_query(c, (2 * 3 * rays + pts) * sizeof(float));
    if (rc)
        return rc;
    float *qo = reinterpret_cast<float *>(c->query_buf), *qd = qo + 3 * rays, *qt = qd + 3 * rays;
    cudaError_t e = launch_density_rays(res, qo, qd, qt, c->stream);
    c->launches++;
    if (e != cudaSuccess)
        return cuda_fail(c, e, "density query rays");
    prenom_ray_batch b{};
    b.obj = obj;
    b.n_rays = (int32_t)rays;
    b.o = qo;
    b.d = qd;
    b.t_in = qt;
    prenom_train_opts op{};
    op.nc = res;
    op.nr = res;
    op.escape_eps = 1e-4f;
    ObjDesc od = make_objdesc(*o, nullptr);
    BatchDesc bd = make_batchdesc(c, *o, b, op, kRender, 128);
    bd.out_sigma = grid_out;
    bd.loss = c->scratch;
    return launch_fused(c, *o, od, bd, PRENOM_KERNEL_RENDER);
}

int prenom_refresh_prior(prenom_ctx *c, int32_t obj, int32_t res)
{
    Object *o = get_obj(c, obj);
    if (!o)
        return fail(c, PRENOM_ERR_INVALID_ARG, "unknown object %d", obj);
    if (res < kMinNr || res > 64)
        return fail(c, PRENOM_ERR_INVALID_ARG, "res must lie in %d..64", kMinNr);
    if (o->R != res) {  // the sampler may still read the old grid: wait for the stream
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "stream");
        cudaFree(o->grid);
        o->grid = nullptr;
        o->R = 0;
        e = cudaMalloc(&o->grid, (size_t)res * res * res * sizeof(float));
        if (e != cudaSuccess)
            return fail(c, PRENOM_ERR_OOM, "prior grid %d^3: %s", res, cudaGetErrorString(e));
        o->R = res;
    }
    // the query renders with given sample depths, so the grid being replaced is never read
    return prenom_density_grid(c, obj, res, o->grid);
}

int prenom_canonical_yaw(prenom_ctx *c, int32_t obj, const float *points, int32_t n_points, int32_t n_gamma,
                         float *scores, int32_t *best)
{
    if (!c)
        return fail(nullptr, PRENOM_ERR_INVALID_ARG, "ctx is NULL");
    Object *o = get_obj(c, obj);
    if (!o)
        return fail(c, PRENOM_ERR_INVALID_ARG, "unknown object %d", obj);
    if (!o->grid)
        return fail(c, PRENOM_ERR_INVALID_ARG, "object %d has no prior grid", obj);
    if (!points || n_points < 1 || n_gamma < 1 || n_gamma > 65536 || !best)
        return fail(c, PRENOM_ERR_INVALID_ARG, "points, n_points >= 1, 1 <= n_gamma <= 65536 and best are required");
    int rc = ensure_query(c, (size_t)n_gamma * sizeof(double));
    if (rc)
        return rc;
    double *d_score = reinterpret_cast<double *>(c->query_buf);
    cudaError_t e = launch_yaw_scores(o->grid, o->R, points, n_points, n_gamma, d_score, c->stream);
    c->launches++;
    if (e != cudaSuccess)
        return cuda_fail(c, e, "yaw score kernel launch");
    std::vector<double> h(n_gamma);
    e = cudaMemcpyAsync(h.data(), d_score, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "yaw scores");
    int b = 0;
    for (int g = 1; g < n_gamma; ++g)
        if (h[g] > h[b])
            b = g;
    *best = b;
    if (scores) {
        std::vector<float> f(h.begin(), h.end());
        e = cudaMemcpy(scores, f.data(), f.size() * sizeof(float), cudaMemcpyDefault);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "yaw scores copy");
    }
    return PRENOM_OK;
}

int prenom_tuning_report(prenom_ctx *c, char *buf, size_t cap)
{
    if (!c || !buf || cap == 0)
        return fail(c, PRENOM_ERR_INVALID_ARG, "ctx, buf and cap are required");
    std::string r;
    for (const auto &kv : c->tune_ms) {
        r += kv.first + ":";
        char tmp[48];
        const bool split_key = kv.first.size() >= 2 && kv.first.compare(kv.first.size() - 2, 2, "/s") == 0;
        for (size_t k = 0; k < kv.second.size(); ++k) {
            snprintf(tmp, sizeof(tmp), " c%d=%.4f", (int)(k % tune_n(split_key)), kv.second[k]);
            r += tmp;
        }
        auto it = c->tune_best.find(kv.first);
        if (it != c->tune_best.end()) {
            snprintf(tmp, sizeof(tmp), " -> c%d", it->second);
            r += tmp;
        }
        r += "\n";
    }
    for (const auto &kv : c->fork_ms) {  // steps of several groups: one after the other / forked
        r += "step " + kv.first + ":";
        char tmp[48];
        for (size_t k = 0; k < kv.second.size(); ++k) {
            snprintf(tmp, sizeof(tmp), " %s=%.4f", k % 2 ? "forked" : "serial", kv.second[k]);
            r += tmp;
        }
        auto it = c->fork_best.find(kv.first);
        if (it != c->fork_best.end())
            r += it->second ? " => forked" : " => serial";
        r += "\n";
    }
    const size_t n = std::min(cap - 1, r.size());
    memcpy(buf, r.data(), n);
    buf[n] = 0;
    return PRENOM_OK;
}

int prenom_zero_grads(prenom_ctx *c, int32_t obj)
{
    Object *o = get_obj(c, obj);
    if (!o)
        return fail(c, PRENOM_ERR_INVALID_ARG, "unknown object %d", obj);
    const cudaError_t e = cudaMemsetAsync(o->grad, 0, (size_t)o->n * sizeof(float), c->stream);
    return e == cudaSuccess ? PRENOM_OK : cuda_fail(c, e, "zero_grads");
}

int prenom_sync(prenom_ctx *c)
{
    if (!c)
        return fail(nullptr, PRENOM_ERR_INVALID_ARG, "ctx is NULL");
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "stream");
    int32_t st = 0;
    e = cudaMemcpy(&st, c->status, sizeof(st), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "status read");
    if (st != 0) {
        cudaMemset(c->status, 0, sizeof(int32_t));
        if (st & kStatusBounds)
            return fail(c, PRENOM_ERR_DEVICE_BOUNDS, "a bounds check of the debug build caught an index outside "
                                                     "its array (the access was skipped)");
        return fail(c, PRENOM_ERR_DEVICE_TIMEOUT, "a kernel gave up waiting for its tensor-core work");
    }
    return PRENOM_OK;
}

int prenom_get_loss_scale(prenom_ctx *c, int32_t obj, float *scale, int32_t *dropped_steps)
{
    Object *o = get_obj(c, obj);
    if (!o)
        return fail(c, PRENOM_ERR_INVALID_ARG, "unknown object %d", obj);
    LossScaleState s{1.f, 0, 0, 0, kLossScaleGrowth, 0, 1.f, 0u, nullptr, 0, 0, 0};
    if (o->lss) {
        cudaError_t e = cudaMemcpyAsync(&s, o->lss, sizeof(s), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "loss-scale read");
    }
    if (scale)
        *scale = s.scale;
    if (dropped_steps)
        *dropped_steps = s.skipped;
    return PRENOM_OK;
}

int prenom_enable_timing(prenom_ctx *c, int32_t enable)
{
    if (!c)
        return fail(nullptr, PRENOM_ERR_INVALID_ARG, "ctx is NULL");
    cudaStreamSynchronize(c->stream);
    for (auto &p : c->pending) {
        c->ev_free.push_back(p.a);
        c->ev_free.push_back(p.b);
    }
    c->pending.clear();
    for (int k = 0; k < PRENOM_N_KERNELS; ++k) {
        c->total_ms[k] = 0.0;
        c->count[k] = 0;
    }
    c->group_time.clear();
    c->timing = enable != 0;
    return PRENOM_OK;
}

int prenom_kernel_time(prenom_ctx *c, int32_t kernel, double *total_ms, int64_t *launches)
{
    if (!c || kernel < 0 || kernel >= PRENOM_N_KERNELS)
        return fail(c, PRENOM_ERR_INVALID_ARG, "bad context or kernel id");
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "stream");
    fold_pending(c);
    if (total_ms)
        *total_ms = c->total_ms[kernel];
    if (launches)
        *launches = c->count[kernel];
    return PRENOM_OK;
}

int prenom_capture_count(prenom_ctx *c, int64_t *captures, int64_t *tuning_calls)
{
    if (!c)
        return fail(nullptr, PRENOM_ERR_INVALID_ARG, "ctx is NULL");
    if (captures)
        *captures = c->n_captures;
    if (tuning_calls)
        *tuning_calls = c->n_tune_calls;
    return PRENOM_OK;
}

int prenom_set_loss_scale(prenom_ctx *c, int32_t obj, float scale, int32_t growth_interval)
{
    Object *o = get_obj(c, obj);
    if (!o)
        return fail(c, PRENOM_ERR_INVALID_ARG, "unknown object %d", obj);
    if (!o->lss)
        return fail(c, PRENOM_ERR_INVALID_ARG, "object %d is FP32: it has no loss scale", obj);
    if (!(scale >= 1.f && scale <= 16777216.f) || growth_interval < 1)
        return fail(c, PRENOM_ERR_INVALID_ARG, "scale must be in [1, 2^24] and growth_interval >= 1");
    const int32_t v[2] = {0, growth_interval};  // good_steps restarts, then the interval
    cudaError_t e = cudaMemcpyAsync(&o->lss->scale, &scale, sizeof(float), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&o->lss->good_steps, &v[0], sizeof(int32_t), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&o->lss->growth_interval, &v[1], sizeof(int32_t), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    return e == cudaSuccess ? PRENOM_OK : cuda_fail(c, e, "loss-scale write");
}

int prenom_timing_report(prenom_ctx *c, char *buf, size_t cap)
{
    if (!c || !buf || cap == 0)
        return fail(c, PRENOM_ERR_INVALID_ARG, "ctx, buf and cap are required");
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "stream");
    fold_pending(c);
    std::string r;
    for (const auto &kv : c->group_time) {
        char tmp[256];
        snprintf(tmp, sizeof(tmp), "%s\tk%d\t%.6f\t%lld\n", c->group_names[kv.first.first].c_str(), kv.first.second,
                 kv.second.first, (long long)kv.second.second);
        r += tmp;
    }
    const size_t n = std::min(cap - 1, r.size());
    memcpy(buf, r.data(), n);
    buf[n] = 0;
    return PRENOM_OK;
}

int prenom_launch_count(prenom_ctx *c, int64_t *launches)
{
    if (!c || !launches)
        return fail(c, PRENOM_ERR_INVALID_ARG, "bad arguments");
    *launches = c->launches;
    return PRENOM_OK;
}

}  // extern "C"
