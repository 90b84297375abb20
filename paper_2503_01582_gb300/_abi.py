"""ctypes binding of include/prenom.h: the same names, argument marshalling only.

Every computation happens inside libprenom.so.  If the library is missing or
cannot be loaded this module raises; there is no fallback path.
"""

from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# PRENOM_DEBUG_BOUNDS=1 in the environment selects the debug build (bounds-checked
# kernels, same entry points), which must have been built.
DEBUG_LIB_PATH = os.path.join(_PKG, "libprenom_debug.so")
LIB_PATH = DEBUG_LIB_PATH if os.environ.get("PRENOM_DEBUG_BOUNDS") == "1" else os.path.join(_PKG, "libprenom.so")

PRENOM_OK = 0
PRENOM_ERR_INVALID_ARG = -1
PRENOM_ERR_OOM = -2
PRENOM_ERR_CUDA = -3
PRENOM_ERR_DEVICE_TIMEOUT = -4
PRENOM_ERR_NONFINITE = -5
PRENOM_ERR_DEVICE_BOUNDS = -6

PRENOM_PRECISION_FP32 = 0
PRENOM_PRECISION_FP16 = 1
PRENOM_PRECISION_BF16 = 2
PRENOM_FEATURES_FP32 = 0
PRENOM_FEATURES_BF16 = 2
PRENOM_FLAG_NO_ADAM = 1
PRENOM_FLAG_CHECK_FINITE = 2
PRENOM_FLAG_NO_GRAPH = 4
PRENOM_FLAG_FUSED = 8
PRENOM_FLAG_SPLIT = 16
PRENOM_FLAG_RETUNE = 32
PRENOM_FLAG_CONCURRENT = 64

PRENOM_STATE_THETA = 0
PRENOM_STATE_GRAD = 1
PRENOM_STATE_ADAM_M = 2
PRENOM_STATE_ADAM_V = 3

PRENOM_KERNEL_TRAIN = 0
PRENOM_KERNEL_ADAM = 1
PRENOM_KERNEL_RENDER = 2
PRENOM_KERNEL_RENDER_BWD = 3
PRENOM_KERNEL_INIT = 4
PRENOM_KERNEL_SAMPLE_ENCODE = 5
PRENOM_KERNEL_SCATTER = 6
PRENOM_N_KERNELS = 7
KERNEL_NAMES = ["train", "adam", "render", "render_bwd", "init", "sample_encode", "scatter"]


class prenom_arch(C.Structure):
    _fields_ = [
        ("L", C.c_int32), ("F", C.c_int32), ("log2T", C.c_int32), ("n_min", C.c_int32), ("n_max", C.c_int32),
        ("width", C.c_int32), ("hidden", C.c_int32), ("precision", C.c_int32),
        ("lambda_d", C.c_float), ("lambda_sigma", C.c_float), ("features", C.c_int32),
    ]


class prenom_keyframe(C.Structure):
    _fields_ = [
        ("width", C.c_int32), ("height", C.c_int32), ("rgb", C.c_void_p), ("depth", C.c_void_p),
        ("mask", C.c_void_p), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
        ("R_wc", C.c_float * 9), ("t_wc", C.c_float * 3),
    ]


class prenom_object_state(C.Structure):
    _fields_ = [("instance", C.c_int32), ("R_wo", C.c_float * 9), ("centre", C.c_float * 3), ("size", C.c_float * 3)]


class prenom_train_opts(C.Structure):
    _fields_ = [
        ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
        ("nc", C.c_int32), ("nr", C.c_int32), ("escape_eps", C.c_float), ("loss_scale_init", C.c_float),
        ("flags", C.c_uint32),
    ]


class prenom_ray_batch(C.Structure):
    _fields_ = [
        ("obj", C.c_int32), ("n_rays", C.c_int32),
        ("o", C.c_void_p), ("d", C.c_void_p), ("rgb", C.c_void_p), ("depth", C.c_void_p),
        ("is_obj", C.c_void_p), ("c_rand", C.c_void_p), ("uniforms", C.c_void_p), ("t_in", C.c_void_p),
    ]


_P = C.c_void_p
_CTX = C.c_void_p
_SIGS = {
    "prenom_create": (C.c_int, [C.POINTER(_CTX), _P, C.c_uint64]),
    "prenom_destroy": (None, [_CTX]),
    "prenom_last_error": (C.c_char_p, [_CTX]),
    "prenom_create_object": (C.c_int, [_CTX, C.POINTER(prenom_arch), _P, C.POINTER(C.c_int32)]),
    "prenom_destroy_object": (C.c_int, [_CTX, C.c_int32]),
    "prenom_param_count": (C.c_int, [_CTX, C.c_int32, C.POINTER(C.c_size_t)]),
    "prenom_arch_param_count": (C.c_int, [C.POINTER(prenom_arch), C.POINTER(C.c_size_t)]),
    "prenom_level_info": (C.c_int, [_CTX, C.c_int32, _P, _P, _P]),
    "prenom_set_prior_grid": (C.c_int, [_CTX, C.c_int32, _P, C.c_int32]),
    "prenom_train_step": (C.c_int, [_CTX, C.POINTER(prenom_ray_batch), C.c_int32,
                                    C.POINTER(prenom_train_opts), _P]),
    "prenom_render": (C.c_int, [_CTX, C.POINTER(prenom_ray_batch), C.POINTER(prenom_train_opts), _P, _P, _P, _P,
                                _P]),
    "prenom_render_backward": (C.c_int, [_CTX, C.POINTER(prenom_ray_batch), C.POINTER(prenom_train_opts), _P, _P]),
    "prenom_get_state": (C.c_int, [_CTX, C.c_int32, C.c_int32, _P, C.c_size_t]),
    "prenom_set_state": (C.c_int, [_CTX, C.c_int32, C.c_int32, _P, C.c_size_t]),
    "prenom_get_step": (C.c_int, [_CTX, C.c_int32, C.POINTER(C.c_int32)]),
    "prenom_set_step": (C.c_int, [_CTX, C.c_int32, C.c_int32]),
    "prenom_zero_grads": (C.c_int, [_CTX, C.c_int32]),
    "prenom_tuning_report": (C.c_int, [_CTX, C.c_char_p, C.c_size_t]),
    "prenom_density_grid": (C.c_int, [_CTX, C.c_int32, C.c_int32, _P]),
    "prenom_make_rays": (C.c_int, [_CTX, C.POINTER(prenom_keyframe), C.c_int32, C.POINTER(prenom_object_state),
                                   C.c_int32, _P, _P, _P, _P, _P, _P, C.POINTER(C.c_int64)]),
    "prenom_refresh_prior": (C.c_int, [_CTX, C.c_int32, C.c_int32]),
    "prenom_canonical_yaw": (C.c_int, [_CTX, C.c_int32, _P, C.c_int32, C.c_int32, _P, C.POINTER(C.c_int32)]),
    "prenom_reptile_begin": (C.c_int, [_CTX, C.c_int32, C.POINTER(C.c_int32), C.c_int32]),
    "prenom_reptile_update": (C.c_int, [_CTX, C.c_int32, C.POINTER(C.c_int32), C.c_int32, C.c_float]),
    "prenom_reptile_task_sum": (C.c_int, [_CTX, C.POINTER(C.c_int32), C.c_int32, _P]),
    "prenom_reptile_apply": (C.c_int, [_CTX, C.c_int32, _P, C.c_int32, C.c_float]),
    "prenom_sync": (C.c_int, [_CTX]),
    "prenom_enable_timing": (C.c_int, [_CTX, C.c_int32]),
    "prenom_kernel_time": (C.c_int, [_CTX, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "prenom_launch_count": (C.c_int, [_CTX, C.POINTER(C.c_int64)]),
    "prenom_get_loss_scale": (C.c_int, [_CTX, C.c_int32, C.POINTER(C.c_float), C.POINTER(C.c_int32)]),
    "prenom_set_loss_scale": (C.c_int, [_CTX, C.c_int32, C.c_float, C.c_int32]),
    "prenom_autotune": (C.c_int, [_CTX, C.POINTER(prenom_ray_batch), C.c_int32, C.POINTER(prenom_train_opts)]),
    "prenom_capture_count": (C.c_int, [_CTX, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "prenom_timing_report": (C.c_int, [_CTX, C.c_char_p, C.c_size_t]),
    "prenom_train_step_noalloc": (C.c_int, [C.POINTER(prenom_arch), _P, _P, _P, C.c_int32, _P, C.c_int32,
                                            C.POINTER(prenom_ray_batch), C.POINTER(prenom_train_opts), _P, _P,
                                            C.c_uint64]),
}

PRENOM_NOALLOC_MAX_PARAMS = 1 << 22

_lib = None


def lib(path: str = LIB_PATH):
    """Loads libprenom.so (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2503_01582_gb300.build.build()")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def symbols():
    """Names of the C-ABI entry points this binding wraps."""
    return list(_SIGS)


class PrenomError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"prenom error {code}: {msg}")
        self.code = code


def check(rc: int, ctx=None):
    if rc != PRENOM_OK:
        msg = lib().prenom_last_error(ctx)
        raise PrenomError(rc, msg.decode() if msg else "")
    return rc


# ---- thin wrappers with the C names (argument marshalling only) ----
def prenom_create(stream: int = 0, seed: int = 0):
    ctx = _CTX()
    check(lib().prenom_create(C.byref(ctx), _P(stream or None), seed))
    return ctx


def prenom_destroy(ctx):
    lib().prenom_destroy(ctx)


def prenom_last_error(ctx) -> str:
    m = lib().prenom_last_error(ctx)
    return m.decode() if m else ""


def prenom_create_object(ctx, arch: prenom_arch, init_params_ptr: int = 0) -> int:
    out = C.c_int32()
    check(lib().prenom_create_object(ctx, C.byref(arch), _P(init_params_ptr or None), C.byref(out)), ctx)
    return out.value


def prenom_destroy_object(ctx, obj: int):
    check(lib().prenom_destroy_object(ctx, obj), ctx)


def prenom_param_count(ctx, obj: int) -> int:
    n = C.c_size_t()
    check(lib().prenom_param_count(ctx, obj, C.byref(n)), ctx)
    return n.value


def prenom_arch_param_count(arch: prenom_arch) -> int:
    n = C.c_size_t()
    check(lib().prenom_arch_param_count(C.byref(arch), C.byref(n)), None)
    return n.value


def prenom_level_info(ctx, obj: int, L: int):
    res = (C.c_int32 * L)()
    off = (C.c_int64 * (L + 1))()
    dense = (C.c_int32 * L)()
    check(lib().prenom_level_info(ctx, obj, C.cast(res, _P), C.cast(off, _P), C.cast(dense, _P)), ctx)
    return list(res), list(off), [bool(x) for x in dense]


def prenom_set_prior_grid(ctx, obj: int, grid_ptr: int, res: int):
    check(lib().prenom_set_prior_grid(ctx, obj, _P(grid_ptr), res), ctx)


def prenom_train_step(ctx, batches, opts: prenom_train_opts, loss_ptr: int = 0):
    arr = (prenom_ray_batch * max(len(batches), 1))(*batches)
    check(lib().prenom_train_step(ctx, arr, len(batches), C.byref(opts), _P(loss_ptr or None)), ctx)


def prenom_render(ctx, batch: prenom_ray_batch, opts: prenom_train_opts, rgb=0, depth=0, acc=0, bins=0, t_out=0):
    check(lib().prenom_render(ctx, C.byref(batch), C.byref(opts), _P(rgb or None), _P(depth or None),
                              _P(acc or None), _P(bins or None), _P(t_out or None)), ctx)


def prenom_render_backward(ctx, batch: prenom_ray_batch, opts: prenom_train_opts, d_out_ptr: int, grad_ptr: int):
    check(lib().prenom_render_backward(ctx, C.byref(batch), C.byref(opts), _P(d_out_ptr or None),
                                       _P(grad_ptr or None)), ctx)


def prenom_get_state(ctx, obj: int, which: int, dst_ptr: int, n: int):
    check(lib().prenom_get_state(ctx, obj, which, _P(dst_ptr), n), ctx)


def prenom_set_state(ctx, obj: int, which: int, src_ptr: int, n: int):
    check(lib().prenom_set_state(ctx, obj, which, _P(src_ptr), n), ctx)


def prenom_get_step(ctx, obj: int) -> int:
    s = C.c_int32()
    check(lib().prenom_get_step(ctx, obj, C.byref(s)), ctx)
    return s.value


def prenom_set_step(ctx, obj: int, step: int):
    check(lib().prenom_set_step(ctx, obj, step), ctx)


def prenom_zero_grads(ctx, obj: int):
    check(lib().prenom_zero_grads(ctx, obj), ctx)


def prenom_tuning_report(ctx) -> str:
    buf = C.create_string_buffer(1 << 16)
    check(lib().prenom_tuning_report(ctx, buf, len(buf)), ctx)
    return buf.value.decode()


def prenom_make_rays(ctx, keyframes, state, n_rays: int, draws_ptr: int, o: int, d: int, rgb: int, depth: int,
                     is_obj: int, want_count: bool) -> int:
    arr = (prenom_keyframe * len(keyframes))(*keyframes)
    cnt = C.c_int64(-1)
    check(lib().prenom_make_rays(ctx, arr, len(keyframes), C.byref(state), n_rays, _P(draws_ptr or None), _P(o),
                                 _P(d), _P(rgb), _P(depth), _P(is_obj), C.byref(cnt) if want_count else None), ctx)
    return cnt.value


def prenom_density_grid(ctx, obj: int, res: int, out_ptr: int):
    check(lib().prenom_density_grid(ctx, obj, res, _P(out_ptr)), ctx)


def prenom_refresh_prior(ctx, obj: int, res: int):
    check(lib().prenom_refresh_prior(ctx, obj, res), ctx)


def prenom_canonical_yaw(ctx, obj: int, points_ptr: int, n_points: int, n_gamma: int, scores_ptr: int) -> int:
    best = C.c_int32()
    check(lib().prenom_canonical_yaw(ctx, obj, _P(points_ptr), n_points, n_gamma, _P(scores_ptr or None),
                                     C.byref(best)), ctx)
    return best.value


def _ids(tasks):
    return (C.c_int32 * len(tasks))(*[int(t) for t in tasks])


def prenom_reptile_begin(ctx, meta: int, tasks):
    check(lib().prenom_reptile_begin(ctx, meta, _ids(tasks), len(tasks)), ctx)


def prenom_reptile_update(ctx, meta: int, tasks, beta: float):
    check(lib().prenom_reptile_update(ctx, meta, _ids(tasks), len(tasks), beta), ctx)


def prenom_reptile_task_sum(ctx, tasks, sum_ptr: int):
    check(lib().prenom_reptile_task_sum(ctx, _ids(tasks), len(tasks), _P(sum_ptr)), ctx)


def prenom_reptile_apply(ctx, meta: int, sum_ptr: int, n_total: int, beta: float):
    check(lib().prenom_reptile_apply(ctx, meta, _P(sum_ptr), n_total, beta), ctx)


def prenom_sync(ctx):
    check(lib().prenom_sync(ctx), ctx)


def prenom_enable_timing(ctx, enable: bool):
    check(lib().prenom_enable_timing(ctx, 1 if enable else 0), ctx)


def prenom_kernel_time(ctx, kernel: int):
    ms = C.c_double()
    n = C.c_int64()
    check(lib().prenom_kernel_time(ctx, kernel, C.byref(ms), C.byref(n)), ctx)
    return ms.value, n.value


def prenom_launch_count(ctx) -> int:
    n = C.c_int64()
    check(lib().prenom_launch_count(ctx, C.byref(n)), ctx)
    return n.value


def prenom_train_step_noalloc(arch: prenom_arch, theta_ptr: int, m_ptr: int, v_ptr: int, step: int, grid_ptr: int,
                              res: int, batch: prenom_ray_batch, opts: prenom_train_opts, loss_ptr: int = 0,
                              stream: int = 0, seed: int = 0):
    """Training step on caller-owned theta / Adam moments that allocates no device memory."""
    check(lib().prenom_train_step_noalloc(C.byref(arch), _P(theta_ptr), _P(m_ptr), _P(v_ptr), step,
                                          _P(grid_ptr or None), res, C.byref(batch), C.byref(opts),
                                          _P(loss_ptr or None), _P(stream or None), seed))


def prenom_get_loss_scale(ctx, obj: int):
    """(current loss scale, steps dropped after a 16-bit overflow) of an object."""
    s = C.c_float()
    n = C.c_int32()
    check(lib().prenom_get_loss_scale(ctx, obj, C.byref(s), C.byref(n)), ctx)
    return s.value, n.value


def prenom_set_loss_scale(ctx, obj: int, scale: float, growth_interval: int = 1000):
    """Loss scale and growth interval (clean steps before it doubles) of a mixed-precision object."""
    check(lib().prenom_set_loss_scale(ctx, obj, scale, growth_interval), ctx)


def prenom_autotune(ctx, batches, opts: prenom_train_opts):
    """The autotuner's calls (gradient-only, cleaned up) and the step graphs, before training."""
    arr = (prenom_ray_batch * max(len(batches), 1))(*batches)
    check(lib().prenom_autotune(ctx, arr, len(batches), C.byref(opts)), ctx)


def prenom_capture_count(ctx):
    """(step graphs captured, steps run as autotuner measurements) so far."""
    a = C.c_int64()
    b = C.c_int64()
    check(lib().prenom_capture_count(ctx, C.byref(a), C.byref(b)), ctx)
    return a.value, b.value


def prenom_timing_report(ctx):
    """Per-group kernel times of timed batched steps: list of (label, kernel id, total ms, launches)."""
    buf = C.create_string_buffer(1 << 16)
    check(lib().prenom_timing_report(ctx, buf, len(buf)), ctx)
    out = []
    for ln in buf.value.decode().splitlines():
        label, k, ms, n = ln.split("\t")
        out.append((label, int(k[1:]), float(ms), int(n)))
    return out
