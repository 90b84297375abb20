"""Analytic scenes, cameras, ray pools and seeded tensors for the PRENOM training step.

Every function takes an explicit seed (or a numpy Generator) and returns numpy
arrays in float32 (inputs of the CUDA path) unless stated otherwise.  Scenes
live in the unit cube [0,1]^3, which plays the role of the normalized object
coordinate space of §III-A; rays are given in that frame with unit-length
directions, so a ray parameter t is a distance in that frame.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

LIGHT_DIR = np.array([1.0, 2.0, 3.0]) / np.sqrt(14.0)


@dataclass
class Primitive:
    """One solid: kind is "sphere" (size = [r]), "box" (size = half extents) or
    "cylinder" (size = [radius, half height], axis = 0/1/2)."""

    kind: str
    centre: np.ndarray
    size: np.ndarray
    albedo: np.ndarray  # [3] or, for a box, optionally [6][3] (one per face)
    axis: int = 2


@dataclass
class Scene:
    prims: list = field(default_factory=list)

    # ---------------------------------------------------------------- geometry
    def sdf(self, p: np.ndarray) -> np.ndarray:
        """Signed distance of the union at points p [..., 3] (exact outside)."""
        d = np.full(p.shape[:-1], np.inf)
        for pr in self.prims:
            q = p - pr.centre
            if pr.kind == "sphere":
                di = np.linalg.norm(q, axis=-1) - pr.size[0]
            elif pr.kind == "box":
                a = np.abs(q) - pr.size
                di = np.linalg.norm(np.maximum(a, 0.0), axis=-1) + np.minimum(a.max(-1), 0.0)
            else:
                ax = pr.axis
                rad = np.sqrt(np.sum(np.delete(q, ax, axis=-1) ** 2, axis=-1))
                a0 = rad - pr.size[0]
                a1 = np.abs(q[..., ax]) - pr.size[1]
                outside = np.sqrt(np.maximum(a0, 0.0) ** 2 + np.maximum(a1, 0.0) ** 2)
                di = outside + np.minimum(np.maximum(a0, a1), 0.0)
            d = np.minimum(d, di)
        return d

    def cast(self, o: np.ndarray, d: np.ndarray):
        """First hit of rays o + t d (d unit) with the union.

        Returns (t [n], normal [n,3], albedo [n,3]); t = inf on a miss.
        """
        n = o.shape[0]
        best_t = np.full(n, np.inf)
        best_nrm = np.zeros((n, 3))
        best_alb = np.zeros((n, 3))
        for pr in self.prims:
            t, nrm, alb = _cast_prim(pr, o, d)
            better = t < best_t
            best_t = np.where(better, t, best_t)
            best_nrm[better] = nrm[better]
            best_alb[better] = alb[better]
        # the object lives in the unit cube: hits outside it do not count
        p = o + np.where(np.isfinite(best_t), best_t, 0.0)[:, None] * d
        inside = np.all((p >= -1e-9) & (p <= 1 + 1e-9), axis=-1)
        best_t = np.where(inside, best_t, np.inf)
        return best_t, best_nrm, best_alb


def _first_positive(t0, t1):
    t = np.where(t0 > 1e-9, t0, np.where(t1 > 1e-9, t1, np.inf))
    return t


def _cast_prim(pr: Primitive, o, d):
    n = o.shape[0]
    alb = np.broadcast_to(np.asarray(pr.albedo, dtype=np.float64).reshape(-1, 3)[0], (n, 3)).copy()
    if pr.kind == "sphere":
        oc = o - pr.centre
        b = np.sum(oc * d, axis=-1)
        c = np.sum(oc * oc, axis=-1) - pr.size[0] ** 2
        disc = b * b - c
        sq = np.sqrt(np.maximum(disc, 0.0))
        t = _first_positive(-b - sq, -b + sq)
        t = np.where(disc >= 0, t, np.inf)
        p = o + np.where(np.isfinite(t), t, 0.0)[:, None] * d
        nrm = (p - pr.centre) / pr.size[0]
        return t, nrm, alb
    if pr.kind == "box":
        lo = pr.centre - pr.size
        hi = pr.centre + pr.size
        with np.errstate(divide="ignore", invalid="ignore"):
            inv = 1.0 / d
            t1 = (lo - o) * inv
            t2 = (hi - o) * inv
        tmin_ax = np.minimum(t1, t2)
        tmax_ax = np.maximum(t1, t2)
        tmin_ax = np.where(np.isnan(tmin_ax), -np.inf, tmin_ax)
        tmax_ax = np.where(np.isnan(tmax_ax), np.inf, tmax_ax)
        tmin = tmin_ax.max(-1)
        tmax = tmax_ax.min(-1)
        hit = (tmax >= np.maximum(tmin, 0.0)) & (tmin > 1e-9)
        t = np.where(hit, tmin, np.inf)
        ax = np.argmax(tmin_ax, axis=-1)
        nrm = np.zeros((n, 3))
        sgn = -np.sign(d[np.arange(n), ax])
        nrm[np.arange(n), ax] = sgn
        albs = np.asarray(pr.albedo, dtype=np.float64).reshape(-1, 3)
        if albs.shape[0] == 6:
            face = ax * 2 + (sgn > 0)
            alb = albs[face]
        return t, nrm, alb
    # cylinder along pr.axis
    ax = pr.axis
    oth = [i for i in range(3) if i != ax]
    oc = o - pr.centre
    r, hh = pr.size
    a = d[:, oth[0]] ** 2 + d[:, oth[1]] ** 2
    b = oc[:, oth[0]] * d[:, oth[0]] + oc[:, oth[1]] * d[:, oth[1]]
    c = oc[:, oth[0]] ** 2 + oc[:, oth[1]] ** 2 - r * r
    with np.errstate(divide="ignore", invalid="ignore"):
        disc = b * b - a * c
        sq = np.sqrt(np.maximum(disc, 0.0))
        ts0 = (-b - sq) / a
        ts1 = (-b + sq) / a
    cands = []
    for ts in (ts0, ts1):
        z = oc[:, ax] + ts * d[:, ax]
        ok = (disc >= 0) & (a > 1e-14) & (np.abs(z) <= hh) & (ts > 1e-9)
        cands.append((np.where(ok, ts, np.inf), 0))
    with np.errstate(divide="ignore", invalid="ignore"):
        for sgn in (-1.0, 1.0):
            tc = (sgn * hh - oc[:, ax]) / d[:, ax]
            px = oc[:, oth[0]] + tc * d[:, oth[0]]
            py = oc[:, oth[1]] + tc * d[:, oth[1]]
            ok = np.isfinite(tc) & (tc > 1e-9) & (px * px + py * py <= r * r)
            cands.append((np.where(ok, tc, np.inf), sgn))
    ts = np.stack([cnd[0] for cnd in cands], axis=-1)
    which = np.argmin(ts, axis=-1)
    t = ts[np.arange(n), which]
    p = oc + np.where(np.isfinite(t), t, 0.0)[:, None] * d
    nrm = np.zeros((n, 3))
    side = which < 2
    nrm[:, oth[0]] = np.where(side, p[:, oth[0]] / r, 0.0)
    nrm[:, oth[1]] = np.where(side, p[:, oth[1]] / r, 0.0)
    capsign = np.where(which == 2, -1.0, 1.0)
    nrm[:, ax] = np.where(side, 0.0, capsign)
    return t, nrm, alb


# ------------------------------------------------------------------ scenes
def scene_sphere_box() -> Scene:
    """Union of a sphere (r 0.3 at (0.38, .5, .5)) and an axis-aligned box
    (half size 0.25 at (0.62, .5, .5)); six fixed face albedos on the box."""
    face_albedo = np.array(
        [
            [0.9, 0.9, 0.2],
            [0.2, 0.8, 0.3],
            [0.2, 0.4, 0.9],
            [0.9, 0.5, 0.1],
            [0.6, 0.2, 0.8],
            [0.3, 0.9, 0.9],
        ]
    )
    return Scene(
        [
            Primitive("sphere", np.array([0.38, 0.5, 0.5]), np.array([0.3]), np.array([0.8, 0.3, 0.2])),
            Primitive("box", np.array([0.62, 0.5, 0.5]), np.array([0.25, 0.25, 0.25]), face_albedo),
        ]
    )


def scene_random_csg(seed: int, scale: float = 1.0) -> Scene:
    """3-6 primitives drawn from {sphere, box, cylinder}; centres in [0.3,0.7]^3,
    sizes in [0.08,0.25] (times `scale`), albedos uniform in [0,1]^3."""
    rng = np.random.default_rng(seed)
    prims = []
    for _ in range(int(rng.integers(3, 7))):
        kind = ["sphere", "box", "cylinder"][int(rng.integers(0, 3))]
        centre = rng.uniform(0.3, 0.7, 3)
        alb = rng.uniform(0.0, 1.0, 3)
        if kind == "sphere":
            size = np.array([rng.uniform(0.08, 0.25)]) * scale
        elif kind == "box":
            size = rng.uniform(0.08, 0.25, 3) * scale
        else:
            size = np.array([rng.uniform(0.08, 0.25), rng.uniform(0.08, 0.25)]) * scale
        prims.append(Primitive(kind, centre, size, alb, axis=int(rng.integers(0, 3))))
    return Scene(prims)


# ----------------------------------------------------------------- cameras
def cameras_on_sphere(n: int, radius: float, fov_deg: float, height: int, width: int, seed: int):
    """n pinhole cameras at random points of a sphere about the cube centre,
    each looking at the centre.  Returns a list of (eye, R_cam_to_world, fy)."""
    rng = np.random.default_rng(seed)
    centre = np.full(3, 0.5)
    cams = []
    for _ in range(n):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        eye = centre + radius * v
        fwd = centre - eye
        fwd /= np.linalg.norm(fwd)
        up = np.array([0.0, 0.0, 1.0]) if abs(fwd[2]) < 0.99 else np.array([0.0, 1.0, 0.0])
        right = np.cross(fwd, up)
        right /= np.linalg.norm(right)
        up2 = np.cross(right, fwd)
        cams.append((eye, np.stack([right, up2, fwd], axis=1), fov_deg, height, width))
    return cams


def _pixel_rays(cam, ys, xs):
    eye, rot, fov_deg, h, w = cam
    th = np.tan(np.deg2rad(fov_deg) * 0.5)
    px = ((xs + 0.5) / w - 0.5) * 2.0 * th * (w / h)
    py = -((ys + 0.5) / h - 0.5) * 2.0 * th
    dirs = np.stack([px, py, np.ones_like(px)], axis=-1) @ rot.T
    dirs /= np.linalg.norm(dirs, axis=-1, keepdims=True)
    o = np.broadcast_to(eye, dirs.shape).copy()
    return o, dirs


def _hits_unit_cube(o, d):
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t1 = (0.0 - o) * inv
        t2 = (1.0 - o) * inv
    tmin = np.where(np.isnan(np.minimum(t1, t2)), -np.inf, np.minimum(t1, t2)).max(-1)
    tmax = np.where(np.isnan(np.maximum(t1, t2)), np.inf, np.maximum(t1, t2)).min(-1)
    return tmax > np.maximum(tmin, 0.0) + 1e-6


@dataclass
class RayPool:
    o: np.ndarray  # [n,3] f32
    d: np.ndarray  # [n,3] f32, unit length
    rgb: np.ndarray  # [n,3] f32 target colour (object rays)
    depth: np.ndarray  # [n] f32 target ray distance (object rays, 0 otherwise)
    is_obj: np.ndarray  # [n] u8, 1 = ray hits the object (R_o), 0 = background (R_b)

    def __len__(self):
        return self.o.shape[0]


def make_ray_pool(scene: Scene, cams, n_rays: int, seed: int, depth_noise: float = 0.0) -> RayPool:
    """Draws pixels uniformly over all cameras, keeps those whose rays enter the
    unit cube, and renders their Lambertian colour and depth analytically."""
    rng = np.random.default_rng(seed)
    os_, ds_ = [], []
    have = 0
    while have < n_rays:
        m = max(4 * (n_rays - have), 1024)
        ci = rng.integers(0, len(cams), m)
        o = np.empty((m, 3))
        d = np.empty((m, 3))
        for k, cam in enumerate(cams):
            sel = np.nonzero(ci == k)[0]
            if sel.size == 0:
                continue
            _, _, _, h, w = cam
            ys = rng.integers(0, h, sel.size).astype(np.float64)
            xs = rng.integers(0, w, sel.size).astype(np.float64)
            o[sel], d[sel] = _pixel_rays(cam, ys, xs)
        keep = _hits_unit_cube(o, d)
        os_.append(o[keep])
        ds_.append(d[keep])
        have += int(keep.sum())
    o = np.concatenate(os_)[:n_rays]
    d = np.concatenate(ds_)[:n_rays]
    t, nrm, alb = scene.cast(o, d)
    hit = np.isfinite(t)
    shade = 0.2 + 0.8 * np.maximum(0.0, nrm @ LIGHT_DIR)
    rgb = np.clip(alb * shade[:, None], 0.0, 1.0)
    rgb = np.where(hit[:, None], rgb, 0.0)
    depth = np.where(hit, t, 0.0)
    if depth_noise > 0:
        depth = np.where(hit, depth + rng.normal(0.0, depth_noise, depth.shape), 0.0)
    return RayPool(
        o.astype(np.float32),
        d.astype(np.float32),
        rgb.astype(np.float32),
        depth.astype(np.float32),
        hit.astype(np.uint8),
    )


# ------------------------------------------------------------ prior grids
def prior_grid(scene: Scene, res: int, seed: int, dilate_voxels: float = 2.0, noise: float = 0.1,
               peak: float = 50.0) -> np.ndarray:
    """Noisy prior density grid [res][res][res] (x fastest) over voxel centres:
    logit +4 inside the shape dilated by `dilate_voxels` voxels, -16 outside,
    plus N(0, noise^2); density = peak * sigmoid(logit)."""
    rng = np.random.default_rng(seed)
    c = (np.arange(res) + 0.5) / res
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    p = np.stack([x, y, z], axis=-1)
    inside = scene.sdf(p) <= dilate_voxels / res
    logit = np.where(inside, 4.0, -16.0) + rng.normal(0.0, noise, inside.shape)
    return (peak / (1.0 + np.exp(-logit))).astype(np.float32)


# ------------------------------------------------------- random draws (inputs)
def stratified_uniforms(n_rays: int, nr: int, seed: int) -> np.ndarray:
    """u[r][k] = (k + xi) / nr with xi ~ U[0,1): sorted along each ray, in [0,1)."""
    rng = np.random.default_rng(seed)
    xi = rng.random((n_rays, nr))
    u = (np.arange(nr)[None, :] + xi) / nr
    return np.minimum(u, np.nextafter(np.float32(1.0), np.float32(0.0))).astype(np.float32)


def random_colours(n_rays: int, seed: int) -> np.ndarray:
    """Background supervision colours C_rand ~ U[0,1)^3 (§III-B, loss)."""
    return np.random.default_rng(seed).random((n_rays, 3)).astype(np.float32)


def init_params(n_hash_params: int, mlp_shapes, seed: int, hash_range: float = 1e-4) -> np.ndarray:
    """Flat initial parameter vector: n_hash_params table values ~ U(-hash_range, hash_range),
    then one row-major (out, in) matrix per entry of mlp_shapes, Xavier-uniform."""
    rng = np.random.default_rng(seed)
    parts = [rng.uniform(-hash_range, hash_range, n_hash_params)]
    for out_f, in_f in mlp_shapes:
        a = np.sqrt(6.0 / (in_f + out_f))
        parts.append(rng.uniform(-a, a, out_f * in_f))
    return np.concatenate(parts).astype(np.float32)


def sample_batch(pool: RayPool, n: int, seed: int) -> dict:
    """n rays drawn uniformly (without replacement) from a pool."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(pool), size=n, replace=False) if n <= len(pool) else rng.integers(0, len(pool), n)
    return dict(
        o=np.ascontiguousarray(pool.o[idx]),
        d=np.ascontiguousarray(pool.d[idx]),
        rgb=np.ascontiguousarray(pool.rgb[idx]),
        depth=np.ascontiguousarray(pool.depth[idx]),
        is_obj=np.ascontiguousarray(pool.is_obj[idx]),
    )


# ------------------------------------------------------------ RGB-D keyframes
def object_pose(centre, yaw: float, size):
    """World placement of the unit-cube scene: p_w = R_wo ((p - 1/2) * size) + centre,
    R_wo a turn by `yaw` about the world z axis."""
    c, s = np.cos(yaw), np.sin(yaw)
    R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    return R, np.asarray(centre, np.float64), np.asarray(size, np.float64)


def keyframe_cameras(n: int, centre, radius: float, seed: int):
    """n camera-to-world poses (R_wc with columns right, down, forward; t_wc) on a
    ring above `centre`, looking at it (pinhole convention: x right, y down)."""
    rng = np.random.default_rng(seed)
    poses = []
    for _ in range(n):
        az = rng.uniform(0.0, 2.0 * np.pi)
        el = rng.uniform(0.2, 0.9)
        eye = np.asarray(centre) + radius * np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])
        fwd = np.asarray(centre) - eye
        fwd /= np.linalg.norm(fwd)
        right = np.cross(fwd, np.array([0.0, 0.0, 1.0]))
        right /= np.linalg.norm(right)
        down = np.cross(fwd, right)
        poses.append((np.stack([right, down, fwd], axis=1), eye))
    return poses


def render_keyframe(scene: Scene, pose, obj, height: int, width: int, fov_deg: float, instance: int,
                    depth_noise: float = 0.0, seed: int = 0) -> dict:
    """RGB (uint8), z-depth (float32, 0 where nothing is hit) and instance mask
    (int32, `instance` on the object, 0 elsewhere) of the scene placed in the
    world by obj = (R_wo, centre, size), seen by a pinhole camera pose = (R_wc, t_wc)."""
    R_wc, t_wc = pose
    R_wo, c, S = obj
    f = 0.5 * height / np.tan(np.deg2rad(fov_deg) * 0.5)
    cx, cy = 0.5 * width, 0.5 * height
    ys, xs = np.mgrid[0:height, 0:width]
    dc = np.stack([(xs + 0.5 - cx) / f, (ys + 0.5 - cy) / f, np.ones_like(xs, dtype=np.float64)], -1).reshape(-1, 3)
    dw = dc @ R_wc.T
    nrm = np.linalg.norm(dw, axis=-1)
    dh = dw / nrm[:, None]
    o_n = ((t_wc - c) @ R_wo) / S + 0.5
    d_n = (dh @ R_wo) / S
    dl = np.linalg.norm(d_n, axis=-1)
    t, nrm_n, alb = scene.cast(np.broadcast_to(o_n, d_n.shape).copy(), d_n / dl[:, None])
    hit = np.isfinite(t)
    t_w = np.where(hit, t / dl, 0.0)  # the object-frame distance back to world units
    n_w = (nrm_n / S) @ R_wo.T  # normals transform with the inverse transpose
    n_w /= np.maximum(np.linalg.norm(n_w, axis=-1, keepdims=True), 1e-12)
    shade = 0.2 + 0.8 * np.maximum(0.0, n_w @ LIGHT_DIR)
    rgb = np.where(hit[:, None], np.clip(alb * shade[:, None], 0.0, 1.0), 0.1)
    z = np.where(hit, t_w / nrm, 0.0)
    if depth_noise > 0:
        z = np.where(hit, z + np.random.default_rng(seed).normal(0.0, depth_noise, z.shape), 0.0)
    return dict(rgb=np.round(rgb * 255).astype(np.uint8).reshape(height, width, 3),
                depth=z.astype(np.float32).reshape(height, width),
                mask=np.where(hit, instance, 0).astype(np.int32).reshape(height, width),
                fx=f, fy=f, cx=cx, cy=cy, R_wc=R_wc.astype(np.float32), t_wc=t_wc.astype(np.float32))
