"""GB300-native training step of PRENOM's object-level NeRFs (arXiv 2503.01582).

The computation lives in libprenom.so (hand-written CUDA for sm_103a behind the
C ABI of include/prenom.h).  This package only marshals torch tensors (device
memory and streams) into that ABI:

    ctx = Context(seed=0)
    obj = ctx.create_object(make_arch(L=16, log2T=19, n_max=2048, width=64))
    ctx.set_prior_grid(obj, grid)                  # [R, R, R] float32
    ctx.train_step([dict(obj=obj, o=o, d=d, rgb=rgb, depth=depth, is_obj=m)],
                   make_opts(nc=64, nr=64, lr=1e-2), loss=loss_buf)
"""

from __future__ import annotations

from . import _abi
from ._abi import (  # noqa: F401
    KERNEL_NAMES,
    PRENOM_ERR_CUDA,
    PRENOM_ERR_DEVICE_TIMEOUT,
    PRENOM_ERR_INVALID_ARG,
    PRENOM_ERR_NONFINITE,
    PRENOM_ERR_OOM,
    PRENOM_FEATURES_BF16,
    PRENOM_FEATURES_FP32,
    PRENOM_FLAG_CHECK_FINITE,
    PRENOM_FLAG_FUSED,
    PRENOM_FLAG_SPLIT,
    PRENOM_FLAG_RETUNE,
    PRENOM_FLAG_CONCURRENT,
    PRENOM_FLAG_NO_ADAM,
    PRENOM_FLAG_NO_GRAPH,
    PRENOM_KERNEL_ADAM,
    PRENOM_KERNEL_RENDER,
    PRENOM_KERNEL_RENDER_BWD,
    PRENOM_KERNEL_SAMPLE_ENCODE,
    PRENOM_KERNEL_SCATTER,
    PRENOM_KERNEL_TRAIN,
    PRENOM_N_KERNELS,
    PRENOM_PRECISION_BF16,
    PRENOM_PRECISION_FP16,
    PRENOM_PRECISION_FP32,
    PRENOM_STATE_ADAM_M,
    PRENOM_STATE_ADAM_V,
    PRENOM_STATE_GRAD,
    PRENOM_STATE_THETA,
    PrenomError,
    prenom_arch,
    prenom_ray_batch,
    prenom_train_opts,
)

__all__ = ["Context", "make_arch", "make_opts", "arch_param_count", "PrenomError"]


def make_arch(L=8, F=2, log2T=14, n_min=16, n_max=256, width=32, hidden=2, precision=PRENOM_PRECISION_FP32,
              lambda_d=0.1, lambda_sigma=0.0, features=0) -> prenom_arch:
    return prenom_arch(L, F, log2T, n_min, n_max, width, hidden, precision, lambda_d, lambda_sigma, features)


def arch_param_count(arch: prenom_arch) -> int:
    """Parameters of an architecture (host query, no context or GPU needed)."""
    return _abi.prenom_arch_param_count(arch)


def make_opts(nc=32, nr=32, lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-15, escape_eps=1e-4, flags=0,
              loss_scale_init=0.0) -> prenom_train_opts:
    return prenom_train_opts(lr, beta1, beta2, eps, nc, nr, escape_eps, loss_scale_init, flags)


def _dptr(t, dtype=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (0 for None)."""
    if t is None:
        return 0
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    return t.data_ptr()


def ray_batch(b: dict) -> prenom_ray_batch:
    """prenom_ray_batch from a dict of CUDA tensors (o, d, rgb, depth, is_obj,
    c_rand, uniforms, t_in; all but o and d optional for rendering)."""
    import torch

    f32, u8 = torch.float32, torch.uint8
    n = int(b["o"].shape[0]) if b.get("o") is not None else int(b.get("n_rays", 0))
    return prenom_ray_batch(
        int(b["obj"]), n,
        _dptr(b.get("o"), f32, "o") or None, _dptr(b.get("d"), f32, "d") or None,
        _dptr(b.get("rgb"), f32, "rgb") or None, _dptr(b.get("depth"), f32, "depth") or None,
        _dptr(b.get("is_obj"), u8, "is_obj") or None, _dptr(b.get("c_rand"), f32, "c_rand") or None,
        _dptr(b.get("uniforms"), f32, "uniforms") or None, _dptr(b.get("t_in"), f32, "t_in") or None,
    )


def _stream_ordered(method):
    """Orders a call's work with torch's current stream: the library's stream
    first waits for the work already queued on the current stream (the call's
    input tensors), and the current stream then waits for the call's work (its
    output tensors), so tensors can be made and read on either stream.  When the
    current stream is the context's own stream both waits are skipped."""
    import functools

    @functools.wraps(method)
    def call(self, *a, **k):
        import torch

        cur = torch.cuda.current_stream()
        other = cur != self.stream
        if other:
            self.stream.wait_stream(cur)
        out = method(self, *a, **k)
        if other:
            cur.wait_stream(self.stream)
        return out

    return call


class Context:
    """One library context on the current CUDA device and a torch stream.
    Every call that launches work is ordered with torch's current stream (see
    _stream_ordered); a loop run under `torch.cuda.stream(context.stream)` skips
    those waits."""

    def __init__(self, seed: int = 0, stream=None):
        import torch

        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._ctx = _abi.prenom_create(self.stream.cuda_stream, seed)
        self._archs = {}

    def close(self):
        if self._ctx is not None:
            _abi.prenom_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- objects ----
    @_stream_ordered
    def create_object(self, arch: prenom_arch, init_params=None) -> int:
        """init_params: None (random), a CUDA float32 tensor or a numpy float32 array."""
        ptr = 0
        keep = None
        if init_params is not None:
            import numpy as np

            if isinstance(init_params, np.ndarray):
                keep = np.ascontiguousarray(init_params, dtype=np.float32)
                ptr = keep.ctypes.data
            else:
                ptr = _dptr(init_params, None, "init_params")
        obj = _abi.prenom_create_object(self._ctx, arch, ptr)
        self._archs[obj] = arch
        del keep
        return obj

    def destroy_object(self, obj: int):
        _abi.prenom_destroy_object(self._ctx, obj)

    def param_count(self, obj: int) -> int:
        return _abi.prenom_param_count(self._ctx, obj)

    def level_info(self, obj: int):
        return _abi.prenom_level_info(self._ctx, obj, self._archs[obj].L)

    @_stream_ordered
    def set_prior_grid(self, obj: int, grid):
        import numpy as np

        if isinstance(grid, np.ndarray):
            g = np.ascontiguousarray(grid, dtype=np.float32)
            _abi.prenom_set_prior_grid(self._ctx, obj, g.ctypes.data, g.shape[0])
            _abi.prenom_sync(self._ctx)
        else:
            _abi.prenom_set_prior_grid(self._ctx, obj, _dptr(grid, None, "grid"), int(grid.shape[0]))

    # ---- steps ----
    @_stream_ordered
    def train_step(self, batches, opts: prenom_train_opts, loss=None):
        cb = [ray_batch(b) for b in batches]
        _abi.prenom_train_step(self._ctx, cb, opts, _dptr(loss, None, "loss"))

    @_stream_ordered
    def render(self, batch: dict, opts: prenom_train_opts, want_samples: bool = False):
        import torch

        n = int(batch["o"].shape[0])
        dev = batch["o"].device
        out = dict(rgb=torch.empty((n, 3), device=dev), depth=torch.empty(n, device=dev),
                   acc=torch.empty(n, device=dev))
        if want_samples:
            out["bins"] = torch.empty((n, opts.nr), dtype=torch.int32, device=dev)
            out["t"] = torch.empty((n, opts.nr), device=dev)
        _abi.prenom_render(self._ctx, ray_batch(batch), opts, out["rgb"].data_ptr(), out["depth"].data_ptr(),
                           out["acc"].data_ptr(), out["bins"].data_ptr() if want_samples else 0,
                           out["t"].data_ptr() if want_samples else 0)
        return out

    @_stream_ordered
    def render_backward(self, batch: dict, opts: prenom_train_opts, d_out, grad):
        _abi.prenom_render_backward(self._ctx, ray_batch(batch), opts, _dptr(d_out, None, "d_out"),
                                    _dptr(grad, None, "grad"))

    # ---- state ----
    @_stream_ordered
    def get_state(self, obj: int, which: int = PRENOM_STATE_THETA):
        import torch

        t = torch.empty(self.param_count(obj), device="cuda")
        _abi.prenom_get_state(self._ctx, obj, which, t.data_ptr(), t.numel())
        return t

    @_stream_ordered
    def set_state(self, obj: int, which: int, src):
        import numpy as np

        if isinstance(src, np.ndarray):
            s = np.ascontiguousarray(src, dtype=np.float32)
            _abi.prenom_set_state(self._ctx, obj, which, s.ctypes.data, s.size)
        else:
            _abi.prenom_set_state(self._ctx, obj, which, _dptr(src, None, "src"), src.numel())

    def get_step(self, obj: int) -> int:
        return _abi.prenom_get_step(self._ctx, obj)

    def set_step(self, obj: int, step: int):
        _abi.prenom_set_step(self._ctx, obj, step)

    def loss_scale(self, obj: int):
        """(current loss scale, steps dropped after a 16-bit overflow)."""
        return _abi.prenom_get_loss_scale(self._ctx, obj)

    def set_loss_scale(self, obj: int, scale: float, growth_interval: int = 1000):
        """Sets a mixed-precision object's loss scale and the clean steps after which it doubles."""
        _abi.prenom_set_loss_scale(self._ctx, obj, scale, growth_interval)

    @_stream_ordered
    def autotune(self, batches, opts: prenom_train_opts):
        """Runs the autotuner's calls for these batches (no Adam, state left as it was) and
        captures the step graphs, so that the following train_step calls only replay."""
        _abi.prenom_autotune(self._ctx, [ray_batch(b) for b in batches], opts)

    def capture_count(self):
        """(step graphs captured, steps run as autotuner measurements) so far."""
        return _abi.prenom_capture_count(self._ctx)

    def timing_report(self):
        """Per-group kernel times of the batched steps timed since enable_timing:
        list of (group label, kernel id, total ms, launches)."""
        return _abi.prenom_timing_report(self._ctx)

    @_stream_ordered
    def zero_grads(self, obj: int):
        _abi.prenom_zero_grads(self._ctx, obj)

    def tuning_report(self) -> str:
        """The autotuner's measured candidates and choices, one line per group signature."""
        return _abi.prenom_tuning_report(self._ctx)

    # ---- training rays from RGB-D keyframes (§III-B "Training Data")
    @_stream_ordered
    def make_rays(self, keyframes, state, n_rays: int, draws=None, count: bool = False):
        """Ray batch (dict of CUDA tensors: o, d, rgb, depth, is_obj) drawn from the
        keyframes' candidate pixels.  keyframes: dicts with CUDA tensors rgb (uint8
        [H,W,3]), depth (float32 [H,W]), mask (int32 [H,W]) and fx, fy, cx, cy,
        R_wc [3,3], t_wc [3]; state: dict(instance, R_wo [3,3], centre [3], size [3]);
        draws: optional CUDA int32/uint32 words [n_rays].  With count=True also returns the
        number of candidates (waits for the stream)."""
        import numpy as np
        import torch

        kfs, keep = [], []
        for k in keyframes:
            rgb, dep, msk = (k["rgb"].contiguous(), k["depth"].contiguous(), k["mask"].contiguous())
            keep += [rgb, dep, msk]
            h, w = dep.shape
            kfs.append(_abi.prenom_keyframe(
                w, h, _dptr(rgb, torch.uint8, "rgb"), _dptr(dep, torch.float32, "depth"),
                _dptr(msk, torch.int32, "mask"), float(k["fx"]), float(k["fy"]), float(k["cx"]), float(k["cy"]),
                (_abi.C.c_float * 9)(*np.asarray(k["R_wc"], np.float32).ravel()),
                (_abi.C.c_float * 3)(*np.asarray(k["t_wc"], np.float32).ravel())))
        st = _abi.prenom_object_state(int(state["instance"]),
                                      (_abi.C.c_float * 9)(*np.asarray(state["R_wo"], np.float32).ravel()),
                                      (_abi.C.c_float * 3)(*np.asarray(state["centre"], np.float32).ravel()),
                                      (_abi.C.c_float * 3)(*np.asarray(state["size"], np.float32).ravel()))
        out = dict(o=torch.empty((n_rays, 3), device="cuda"), d=torch.empty((n_rays, 3), device="cuda"),
                   rgb=torch.empty((n_rays, 3), device="cuda"), depth=torch.empty(n_rays, device="cuda"),
                   is_obj=torch.empty(n_rays, dtype=torch.uint8, device="cuda"))
        if draws is not None and (draws.is_floating_point() or draws.element_size() != 4):
            raise TypeError("draws must hold 32-bit integer words (int32 or uint32)")
        n = _abi.prenom_make_rays(self._ctx, kfs, st, n_rays, _dptr(draws, None, "draws"), out["o"].data_ptr(),
                                  out["d"].data_ptr(), out["rgb"].data_ptr(), out["depth"].data_ptr(),
                                  out["is_obj"].data_ptr(), count)
        del keep
        return (out, n) if count else out

    # ---- prior density grid (§III-A mesh generation, §III-B refresh) and Eq. 3
    @_stream_ordered
    def density_grid(self, obj: int, res: int):
        """[res, res, res] (z, y, x) CUDA tensor: the field's density at the voxel centres."""
        import torch

        out = torch.empty((res, res, res), device="cuda")
        _abi.prenom_density_grid(self._ctx, obj, res, out.data_ptr())
        return out

    @_stream_ordered
    def refresh_prior(self, obj: int, res: int):
        """Replaces the object's prior grid by its own density at resolution res."""
        _abi.prenom_refresh_prior(self._ctx, obj, res)

    @_stream_ordered
    def canonical_yaw(self, obj: int, points, n_gamma: int):
        """Eq. 3 with the object's prior grid: (best yaw index, scores [n_gamma])."""
        import torch

        scores = torch.empty(n_gamma, device="cuda")
        best = _abi.prenom_canonical_yaw(self._ctx, obj, _dptr(points, torch.float32, "points"), points.shape[0],
                                         n_gamma, scores.data_ptr())
        return best, scores

    # ---- Reptile meta step (§III-A, Eq. 1-2)
    @_stream_ordered
    def reptile_begin(self, meta: int, tasks):
        """Every task object <- the meta object's parameters, fresh Adam state."""
        _abi.prenom_reptile_begin(self._ctx, meta, list(tasks))

    @_stream_ordered
    def reptile_update(self, meta: int, tasks, beta: float):
        """theta_meta <- theta_meta + beta (mean of the tasks' parameters - theta_meta)."""
        _abi.prenom_reptile_update(self._ctx, meta, list(tasks), beta)

    @_stream_ordered
    def reptile_task_sum(self, tasks, out):
        """out (CUDA float32, param_count) <- sum of the tasks' parameters."""
        _abi.prenom_reptile_task_sum(self._ctx, list(tasks), _dptr(out, name="out"))

    @_stream_ordered
    def reptile_apply(self, meta: int, task_sum, n_total: int, beta: float):
        """theta_meta <- theta_meta + beta (task_sum / n_total - theta_meta)."""
        _abi.prenom_reptile_apply(self._ctx, meta, _dptr(task_sum, name="task_sum"), n_total, beta)

    def sync(self):
        _abi.prenom_sync(self._ctx)

    # ---- instrumentation ----
    def enable_timing(self, on: bool = True):
        _abi.prenom_enable_timing(self._ctx, on)

    def kernel_time(self, kernel: int):
        """(total ms, launches) since timing was enabled."""
        return _abi.prenom_kernel_time(self._ctx, kernel)

    def launch_count(self) -> int:
        return _abi.prenom_launch_count(self._ctx)
