"""FP64 CPU oracle of the PRENOM object-NeRF training step (arXiv 2503.01582).

TEST INFRASTRUCTURE ONLY.  The tests, the package smoke check and the
benchmark's CPU-baseline leg are its only users; the product path never
imports it.  It shares no code with the CUDA library: the arithmetic lives in
prenom_oracle.c (plain C, double precision, sequential) and this module only
marshals numpy arrays into it.

Section and equation numbers refer to the paper: §III-B "Probabilistic Ray
Sampling" (Eq. 4 occupancy, Eq. 5 termination probability, Eq. 6 CDF),
"Volume Rendering" (Eq. 7), the losses (Eq. 8, Eq. 9) and Adam.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prenom_oracle.c")
_HDR = os.path.join(_HERE, "prenom_oracle.h")
_LIB = os.path.join(_HERE, "liboracle_prenom.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (-O2, no fast-math, no FP contraction)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR)
    )
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
             "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class _Arch(C.Structure):
    _fields_ = [
        ("L", C.c_int), ("F", C.c_int), ("log2T", C.c_int), ("n_min", C.c_int), ("n_max", C.c_int),
        ("width", C.c_int), ("hidden", C.c_int), ("lambda_d", C.c_double), ("lambda_sigma", C.c_double),
    ]


@dataclass(frozen=True)
class Arch:
    """Architecture alpha of one object NeRF (hash grid + MLP + loss weights)."""

    L: int = 8
    F: int = 2
    log2T: int = 14
    n_min: int = 16
    n_max: int = 256
    width: int = 32
    hidden: int = 2
    lambda_d: float = 0.1
    lambda_sigma: float = 0.0

    def c(self) -> _Arch:
        return _Arch(self.L, self.F, self.log2T, self.n_min, self.n_max, self.width, self.hidden,
                     self.lambda_d, self.lambda_sigma)

    @property
    def n_in(self) -> int:
        return self.L * self.F

    def mlp_shapes(self):
        shapes = [(self.width, self.n_in)]
        shapes += [(self.width, self.width)] * (self.hidden - 1)
        shapes += [(4, self.width)]
        return shapes


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_F = C.POINTER(C.c_float)
_U8 = C.POINTER(C.c_uint8)
_U32 = C.POINTER(C.c_uint32)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        A = C.POINTER(_Arch)
        sig = {
            "orc_level_res": (C.c_int, [A, C.c_int]),
            "orc_level_dense": (C.c_int, [A, C.c_int]),
            "orc_level_entries": (C.c_int64, [A, C.c_int]),
            "orc_level_offset": (C.c_int64, [A, C.c_int]),
            "orc_n_hash_params": (C.c_int64, [A]),
            "orc_n_mlp_params": (C.c_int64, [A]),
            "orc_param_count": (C.c_int64, [A]),
            "orc_mlp_offset": (C.c_int64, [A, C.c_int]),
            "orc_grid_index": (C.c_uint32, [A, C.c_int, C.c_uint32, C.c_uint32, C.c_uint32]),
            "orc_ray_box": (C.c_int, [_D, _D, _D, _D]),
            "orc_prior_lookup": (C.c_double, [_D, C.c_int, _D]),
            "orc_cdf_invert": (None, [_D, C.c_int, _D, C.c_int, C.c_double, C.c_double, _I, _D]),
            "orc_sample_ray": (C.c_int, [_D, C.c_int, _D, _D, C.c_int, C.c_int, C.c_double, _D,
                                         _D, _D, _D, _I, _D, _D, _D]),
            "orc_encode": (None, [A, _D, _D, _D]),
            "orc_encode_backward": (None, [A, _D, _D, _D]),
            "orc_mlp_forward": (None, [A, _D, _D, _D, _D]),
            "orc_mlp_backward": (None, [A, _D, _D, _D, _D, _D, _D]),
            "orc_composite": (None, [C.c_int, _D, _D, _D, C.c_double, _D, _D, _D, _D]),
            "orc_composite_backward": (None, [C.c_int, _D, _D, _D, C.c_double, _D, C.c_double,
                                              C.c_double, _D, _D]),
            "orc_ray_loss": (C.c_double, [C.c_int, _D, C.c_double, C.c_double, _D, C.c_double, _D,
                                          C.c_double, _D, _D, _D]),
            "orc_batch": (C.c_double, [A, _D, _D, C.c_int, C.c_int, _D, _D, _D, _D, _U8, _D, _D, _D,
                                       C.c_int, C.c_int, C.c_double, _D, _D, _D, _D, _I, _D, _D, _D]),
            "orc_adam": (None, [C.c_int64, _D, _D, _D, _D, C.c_int, C.c_double, C.c_double,
                                C.c_double, C.c_double]),
            "orc_philox4x32_10": (None, [_U32, _U32, _U32]),
            "orc_reptile": (None, [C.c_int64, _D, C.POINTER(_D), C.c_int, C.c_double]),
            "orc_density_grid": (None, [A, _D, C.c_int, _D]),
            "orc_make_rays": (C.c_int64, [C.POINTER(_Keyframe), C.c_int, C.POINTER(_ObjState), C.c_int,
                                          C.POINTER(C.c_uint32), _F, _F, _F, _F, C.POINTER(C.c_uint8)]),
            "orc_canonical_yaw": (C.c_int, [_D, C.c_int, _D, C.c_int, C.c_int, _D]),
            "orc_philox_uniforms": (None, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, C.c_int, _F]),
            "orc_philox_colours": (None, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, _F]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _d(x):
    """float64, C-contiguous copy/view of x (or None)."""
    if x is None:
        return None
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _p(x, ty=_D):
    return None if x is None else x.ctypes.data_as(ty)


# ------------------------------------------------------------------ geometry
def level_res(a: Arch, l: int) -> int:
    return lib().orc_level_res(C.byref(a.c()), l)


def level_dense(a: Arch, l: int) -> bool:
    return bool(lib().orc_level_dense(C.byref(a.c()), l))


def level_entries(a: Arch, l: int) -> int:
    return lib().orc_level_entries(C.byref(a.c()), l)


def level_offset(a: Arch, l: int) -> int:
    return lib().orc_level_offset(C.byref(a.c()), l)


def n_hash_params(a: Arch) -> int:
    return lib().orc_n_hash_params(C.byref(a.c()))


def n_mlp_params(a: Arch) -> int:
    return lib().orc_n_mlp_params(C.byref(a.c()))


def param_count(a: Arch) -> int:
    return lib().orc_param_count(C.byref(a.c()))


def mlp_offset(a: Arch, layer: int) -> int:
    return lib().orc_mlp_offset(C.byref(a.c()), layer)


def grid_index(a: Arch, l: int, cx: int, cy: int, cz: int) -> int:
    return lib().orc_grid_index(C.byref(a.c()), l, cx, cy, cz)


# ------------------------------------------------------------------ sampling
def ray_box(o, d):
    o, d = _d(o), _d(d)
    tn, tf = C.c_double(), C.c_double()
    hit = lib().orc_ray_box(_p(o), _p(d), C.byref(tn), C.byref(tf))
    return bool(hit), tn.value, tf.value


def prior_lookup(grid, x) -> float:
    g = _d(grid)
    return lib().orc_prior_lookup(_p(g), g.shape[0], _p(_d(x)))


def cdf_invert(cdf, u, tn: float, tf: float):
    cdf, u = _d(cdf), _d(u)
    nc, nr = cdf.size - 1, u.size
    bins = np.zeros(nr, dtype=np.int32)
    t = np.zeros(nr)
    lib().orc_cdf_invert(_p(cdf), nc, _p(u), nr, tn, tf, _p(bins, _I), _p(t))
    return bins, t


def _need(x, size: int, name: str):
    """The C routines read exactly `size` values of an optional array: a shorter
    (or longer) one is a caller's mistake, reported here instead of read past."""
    if x is not None and x.size != size:
        raise ValueError(f"{name} has {x.size} values, {size} expected")


def sample_ray(grid, o, d, nc: int, nr: int, eps: float, u):
    g, o, d, u = _d(grid), _d(o), _d(d), _d(u)
    _need(u, nr, "u")
    out = dict(probe_sigma=np.zeros(nc), rho_term=np.zeros(nc), cdf=np.zeros(nc + 1),
               bins=np.zeros(nr, dtype=np.int32), t=np.zeros(nr))
    tn, tf = C.c_double(), C.c_double()
    esc = lib().orc_sample_ray(_p(g), g.shape[0], _p(o), _p(d), nc, nr, eps, _p(u),
                               _p(out["probe_sigma"]), _p(out["rho_term"]), _p(out["cdf"]),
                               _p(out["bins"], _I), _p(out["t"]), C.byref(tn), C.byref(tf))
    out.update(escape=bool(esc), tn=tn.value, tf=tf.value)
    return out


# --------------------------------------------------------------------- field
def encode(a: Arch, theta, p):
    theta, p = _d(theta), _d(p)
    enc = np.zeros(a.n_in)
    lib().orc_encode(C.byref(a.c()), _p(theta), _p(p), _p(enc))
    return enc


def encode_backward(a: Arch, p, denc, n_params: int):
    grad = np.zeros(n_params)
    lib().orc_encode_backward(C.byref(a.c()), _p(_d(p)), _p(_d(denc)), _p(grad))
    return grad


def mlp_forward(a: Arch, theta, enc):
    theta, enc = _d(theta), _d(enc)
    acts = np.zeros(a.hidden * a.width)
    out = np.zeros(4)
    lib().orc_mlp_forward(C.byref(a.c()), _p(theta), _p(enc), _p(acts), _p(out))
    return acts, out


def mlp_backward(a: Arch, theta, enc, acts, dout):
    theta = _d(theta)
    grad = np.zeros(theta.size)
    denc = np.zeros(a.n_in)
    lib().orc_mlp_backward(C.byref(a.c()), _p(theta), _p(_d(enc)), _p(_d(acts)), _p(_d(dout)),
                           _p(grad), _p(denc))
    return grad, denc


# ----------------------------------------------------------------- rendering
def composite(sigma, c, t, tf: float):
    sigma, c, t = _d(sigma), _d(c), _d(t)
    nr = sigma.size
    w = np.zeros(nr)
    Cc = np.zeros(3)
    D, A = C.c_double(), C.c_double()
    lib().orc_composite(nr, _p(sigma), _p(c), _p(t), tf, _p(w), _p(Cc), C.byref(D), C.byref(A))
    return w, Cc, D.value, A.value


def composite_backward(sigma, c, t, tf: float, gC, gD: float, gA: float):
    sigma, c, t = _d(sigma), _d(c), _d(t)
    nr = sigma.size
    ds = np.zeros(nr)
    dc = np.zeros((nr, 3))
    lib().orc_composite_backward(nr, _p(sigma), _p(c), _p(t), tf, _p(_d(gC)), gD, gA, _p(ds), _p(dc))
    return ds, dc


def ray_loss(is_obj: bool, Cc, D: float, A: float, Cgt, Dgt: float, crand, lambda_d: float):
    gC = np.zeros(3)
    gD, gA = C.c_double(), C.c_double()
    crand = _d(crand if crand is not None else np.zeros(3))
    L = lib().orc_ray_loss(int(is_obj), _p(_d(Cc)), D, A, _p(_d(Cgt)), Dgt, _p(crand), lambda_d,
                           _p(gC), C.byref(gD), C.byref(gA))
    return L, gC, gD.value, gA.value


def batch(a: Arch, theta, grid, rays: dict, nc: int, nr: int, eps: float = 1e-4, *, u=None,
          t_in=None, c_rand=None, upstream=None, want_grad: bool = False, want_samples: bool = True):
    """Forward (and optionally backward) of one object's ray batch.

    rays: dict with o [n,3], d [n,3], rgb [n,3], depth [n], is_obj [n] (u8).
    Returns dict(loss, rgb, depth, acc, bins, t, sigma, grad)."""
    theta = _d(theta)
    g = _d(grid)
    n = int(np.asarray(rays["o"]).shape[0])
    o, d = _d(rays["o"]), _d(rays["d"])
    rgb = _d(rays.get("rgb", np.zeros((n, 3))))
    depth = _d(rays.get("depth", np.zeros(n)))
    is_obj = np.ascontiguousarray(np.asarray(rays.get("is_obj", np.ones(n)), dtype=np.uint8))
    u = _d(u)
    t_in = _d(t_in)
    c_rand = _d(c_rand)
    upstream = _d(upstream)
    for x, size, name in ((u, n * nr, "u"), (t_in, n * nr, "t_in"), (c_rand, n * 3, "c_rand"),
                          (upstream, n * 5, "upstream"), (theta, param_count(a), "theta")):
        _need(x, size, name)
    out = dict(rgb=np.zeros((n, 3)), depth=np.zeros(n), acc=np.zeros(n))
    if want_samples:
        out.update(bins=np.zeros((n, nr), dtype=np.int32), t=np.zeros((n, nr)), sigma=np.zeros((n, nr)))
    grad = np.zeros(theta.size) if want_grad else None
    loss = lib().orc_batch(
        C.byref(a.c()), _p(theta), _p(g), 0 if g is None else g.shape[0], n, _p(o), _p(d), _p(rgb),
        _p(depth), _p(is_obj, _U8), _p(c_rand), _p(u), _p(t_in), nc, nr, eps, _p(upstream),
        _p(out["rgb"]), _p(out["depth"]), _p(out["acc"]), _p(out.get("bins"), _I), _p(out.get("t")),
        _p(out.get("sigma")), _p(grad))
    out["loss"] = loss
    out["grad"] = grad
    return out


def adam(theta, m, v, g, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.99,
         eps: float = 1e-15):
    """In-place dense Adam on float64 arrays."""
    for x in (theta, m, v):
        assert x.dtype == np.float64 and x.flags.c_contiguous
    g = _d(g)
    lib().orc_adam(theta.size, _p(theta), _p(m), _p(v), _p(g), step, lr, beta1, beta2, eps)


class _Keyframe(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("rgb", C.POINTER(C.c_uint8)), ("depth", C.POINTER(C.c_float)),
                ("mask", C.POINTER(C.c_int32)), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("R_wc", C.c_float * 9), ("t_wc", C.c_float * 3)]


class _ObjState(C.Structure):
    _fields_ = [("instance", C.c_int), ("R_wo", C.c_float * 9), ("centre", C.c_float * 3), ("size", C.c_float * 3)]


def make_rays(keyframes, state, draws):
    """Training rays from RGB-D keyframes (§III-B "Training Data").  keyframes:
    dicts with rgb uint8 [H,W,3], depth float32 [H,W], mask int32 [H,W], fx, fy,
    cx, cy, R_wc [3,3], t_wc [3]; state: dict(instance, R_wo [3,3], centre [3],
    size [3]); draws: uint32 [n].  Returns (rays dict, number of candidates)."""
    keep = []
    arr = (_Keyframe * max(len(keyframes), 1))()
    for i, k in enumerate(keyframes):
        rgb = np.ascontiguousarray(k["rgb"], np.uint8)
        dep = np.ascontiguousarray(k["depth"], np.float32)
        msk = np.ascontiguousarray(k["mask"], np.int32)
        keep += [rgb, dep, msk]
        h, w = dep.shape
        arr[i] = _Keyframe(w, h, rgb.ctypes.data_as(C.POINTER(C.c_uint8)), dep.ctypes.data_as(C.POINTER(C.c_float)),
                           msk.ctypes.data_as(C.POINTER(C.c_int32)), k["fx"], k["fy"], k["cx"], k["cy"],
                           (C.c_float * 9)(*np.asarray(k["R_wc"], np.float32).ravel()),
                           (C.c_float * 3)(*np.asarray(k["t_wc"], np.float32).ravel()))
    st = _ObjState(int(state["instance"]), (C.c_float * 9)(*np.asarray(state["R_wo"], np.float32).ravel()),
                   (C.c_float * 3)(*np.asarray(state["centre"], np.float32).ravel()),
                   (C.c_float * 3)(*np.asarray(state["size"], np.float32).ravel()))
    dr = np.ascontiguousarray(draws, np.uint32)
    n = dr.size
    o = np.zeros((n, 3), np.float32)
    d = np.zeros((n, 3), np.float32)
    rgb = np.zeros((n, 3), np.float32)
    depth = np.zeros(n, np.float32)
    is_obj = np.zeros(n, np.uint8)
    f = lambda a: a.ctypes.data_as(_F)  # noqa: E731
    count = lib().orc_make_rays(arr, len(keyframes), C.byref(st), n, dr.ctypes.data_as(C.POINTER(C.c_uint32)), f(o),
                                f(d), f(rgb), f(depth), is_obj.ctypes.data_as(C.POINTER(C.c_uint8)))
    return dict(o=o, d=d, rgb=rgb, depth=depth, is_obj=is_obj), int(count)


def density_grid(a: Arch, theta, R: int):
    """[R, R, R] (z, y, x) density of the field at the voxel centres."""
    th = _d(theta)
    out = np.zeros((R, R, R))
    lib().orc_density_grid(C.byref(a.c()), _p(th), R, _p(out))
    return out


def canonical_yaw(grid, P, n_gamma: int):
    """Eq. 3: (index of the best yaw sample, scores of all n_gamma samples)."""
    g = _d(grid)
    R = g.shape[0]
    pts = _d(np.asarray(P).reshape(-1, 3))
    score = np.zeros(n_gamma)
    best = lib().orc_canonical_yaw(_p(g), R, _p(pts), pts.shape[0], n_gamma, _p(score))
    return best, score


def reptile(theta, tasks, beta: float):
    """In-place Reptile outer update (Eq. 2, batched over the tasks) of a float64 array."""
    assert theta.dtype == np.float64 and theta.flags.c_contiguous
    ts = [_d(t) for t in tasks]
    assert all(t.size == theta.size for t in ts) and len(ts) > 0
    arr = (_D * len(ts))(*[_p(t) for t in ts])
    lib().orc_reptile(theta.size, _p(theta), arr, len(ts), beta)


def meta_step(a: Arch, theta_meta, grid_of, task_batches, nc: int, nr: int, *, lr: float = 1e-2,
              beta: float = 0.1, **kw):
    """One meta-training step (§III-A): every task starts from theta_meta with fresh
    Adam state, takes len(task_batches[t]) inner steps (Eq. 1, with Adam as the inner
    optimiser) on its own batches and prior grid, then Eq. 2 moves theta_meta toward
    the tasks' mean.  task_batches[t] is a list of dicts (rays plus optional
    t_in / u / c_rand).  Returns the new theta_meta and each task's losses."""
    theta = _d(theta_meta).copy()
    finals, losses = [], []
    for t, batches in enumerate(task_batches):
        ob = OracleObject(a, theta, grid_of(t))
        lt = []
        for b in batches:
            rays = {k: b[k] for k in ("o", "d", "rgb", "depth", "is_obj")}
            lt.append(ob.train_step(rays, nc, nr, u=b.get("u"), t_in=b.get("t_in"), c_rand=b.get("c_rand"), lr=lr,
                                    **kw))
        finals.append(ob.theta)
        losses.append(lt)
    reptile(theta, finals, beta)
    return theta, losses


# -------------------------------------------------------------------- Philox
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, _U32), _p(k, _U32), _p(out, _U32))
    return out


def philox_uniforms(seed: int, step: int, obj: int, n: int, nr: int):
    u = np.zeros((n, nr), dtype=np.float32)
    lib().orc_philox_uniforms(seed, step, obj, n, nr, _p(u, _F))
    return u


def philox_colours(seed: int, step: int, obj: int, n: int):
    c = np.zeros((n, 3), dtype=np.float32)
    lib().orc_philox_colours(seed, step, obj, n, _p(c, _F))
    return c


# ---------------------------------------------------------- training object
class OracleObject:
    """One object's FP64 state (theta, Adam m, v, step) trained by the oracle."""

    def __init__(self, a: Arch, theta0, grid):
        self.a = a
        self.theta = _d(theta0).copy()
        self.m = np.zeros_like(self.theta)
        self.v = np.zeros_like(self.theta)
        self.step = 0
        self.grid = _d(grid)

    def train_step(self, rays: dict, nc: int, nr: int, *, u=None, t_in=None, c_rand=None,
                   lr: float = 1e-2, beta1: float = 0.9, beta2: float = 0.99, eps: float = 1e-15,
                   escape_eps: float = 1e-4) -> float:
        out = batch(self.a, self.theta, self.grid, rays, nc, nr, escape_eps, u=u, t_in=t_in,
                    c_rand=c_rand, want_grad=True, want_samples=False)
        self.step += 1
        adam(self.theta, self.m, self.v, out["grad"], self.step, lr, beta1, beta2, eps)
        return out["loss"]
