"""Shared seeded cases for the tests (inputs from synth/, expectations from oracle/)."""

from __future__ import annotations

import numpy as np

import oracle as orc
from synth import (cameras_on_sphere, init_params, make_ray_pool, prior_grid, random_colours, sample_batch,
                   scene_random_csg, scene_sphere_box, stratified_uniforms)

CFG1 = dict(L=8, F=2, log2T=14, n_min=16, n_max=256, width=32, hidden=2, lambda_d=0.1, lambda_sigma=0.0)
CFG2 = dict(L=16, F=2, log2T=19, n_min=16, n_max=2048, width=64, hidden=2, lambda_d=0.1, lambda_sigma=0.0)

_POOLS = {}


def pool_cfg1(n=8192):
    key = ("cfg1", n)
    if key not in _POOLS:
        sc = scene_sphere_box()
        _POOLS[key] = (sc, make_ray_pool(sc, cameras_on_sphere(8, 2.0, 40, 64, 64, 0), n, 0))
    return _POOLS[key]


def pool_cfg2(n=16384, seed=0):
    key = ("cfg2", n, seed)
    if key not in _POOLS:
        sc = scene_random_csg(seed)
        _POOLS[key] = (sc, make_ray_pool(sc, cameras_on_sphere(24, 2.0, 50, 480, 640, seed), n, seed,
                                         depth_noise=0.004))
    return _POOLS[key]


def case(arch: dict, n_rays: int, nr: int, nc: int, seed: int = 1, grid_res: int = 32, hash_range: float = 0.05,
         scene: str = "cfg1"):
    """One seeded case: oracle Arch, theta0, grid, rays, uniforms, colours."""
    a = orc.Arch(**arch)
    sc, pool = pool_cfg1() if scene == "cfg1" else pool_cfg2()
    rays = sample_batch(pool, n_rays, seed)
    grid = prior_grid(sc, grid_res, seed)
    u = stratified_uniforms(n_rays, nr, seed + 1)
    cr = random_colours(n_rays, seed + 2)
    theta = init_params(orc.n_hash_params(a), a.mlp_shapes(), seed + 3, hash_range=hash_range)
    return a, theta, grid, rays, u, cr


def rel(x, y) -> float:
    """max |x - y| / max |y| over the tensor (the acceptance measure)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    den = np.max(np.abs(y)) if y.size else 0.0
    if den == 0.0:
        return float(np.max(np.abs(x))) if x.size else 0.0
    return float(np.max(np.abs(x - y)) / den)


def oracle_samples(grid, rays, u, nc, nr, eps=1e-4):
    """Per-ray oracle sampler outputs: cdf [n][nc+1], bins [n][nr], t [n][nr], escape [n], tn, tf."""
    n = u.shape[0]
    out = dict(cdf=np.zeros((n, nc + 1)), bins=np.zeros((n, nr), np.int32), t=np.zeros((n, nr)),
               escape=np.zeros(n, bool), tn=np.zeros(n), tf=np.zeros(n))
    for r in range(n):
        s = orc.sample_ray(grid, rays["o"][r], rays["d"][r], nc, nr, eps, u[r])
        out["cdf"][r] = s["cdf"]
        out["bins"][r] = s["bins"]
        out["t"][r] = s["t"]
        out["escape"][r] = s["escape"]
        out["tn"][r] = s["tn"]
        out["tf"][r] = s["tf"]
    return out


def oracle_t(grid, rays, u, nc, nr, eps=1e-4):
    """The oracle's sample depths rounded to FP32: fed as t_in to both sides so
    that encoding, MLP, rendering and gradients are compared on identical
    samples.  (The FP32 inverse CDF places a sample in a bin of mass m only to
    ~1e-7 / m of the bin width, which the fine levels turn into weight errors;
    the sampler is compared separately, with that bound.)"""
    return oracle_samples(grid, rays, u, nc, nr, eps)["t"].astype(np.float32)


def conditioned_uniforms(grid, rays, nc, nr, seed, min_mass=0.02, eps=1e-4):
    """Stratified uniforms re-drawn, inside their own stratum, away from bins
    whose oracle mass is below min_mass (where FP32 inversion is ill-conditioned).
    Samples whose whole stratum lies in such bins keep their draw."""
    rng = np.random.default_rng(seed)
    u = stratified_uniforms(rays["o"].shape[0], nr, seed).astype(np.float64)
    for r in range(u.shape[0]):
        cdf = orc.sample_ray(grid, rays["o"][r], rays["d"][r], nc, nr, eps, u[r].astype(np.float32))["cdf"]
        mass = np.diff(cdf)
        for k in range(nr):
            b = min(int(np.searchsorted(cdf[1:], u[r, k], side="right")), nc - 1)
            if mass[b] >= min_mass:
                continue
            lo_s, hi_s = k / nr, (k + 1) / nr
            good = [(max(cdf[i], lo_s), min(cdf[i + 1], hi_s)) for i in range(nc)
                    if mass[i] >= min_mass and min(cdf[i + 1], hi_s) - max(cdf[i], lo_s) > 1e-6]
            if good:
                lo, hi = good[int(rng.integers(0, len(good)))]
                u[r, k] = lo + (hi - lo) * (0.05 + 0.9 * rng.random())
    return np.minimum(u, np.nextafter(np.float32(1), np.float32(0))).astype(np.float32)


def bins_match(gpu_bins, want_bins, cdf_rows, u, margin=1e-5):
    """Bin indices must equal the oracle's wherever the uniform is farther than
    `margin` from every FP64 CDF edge; inside the margin the GPU's bin must
    still bracket u up to the margin.  Returns (mismatches, samples near an edge)."""
    bad = 0
    near = 0
    for r in range(u.shape[0]):
        cdf = cdf_rows[r]
        for k in range(u.shape[1]):
            b = int(gpu_bins[r, k])
            if np.min(np.abs(cdf - u[r, k])) > margin:
                bad += int(b != int(want_bins[r, k]))
            else:
                near += 1
                ok = 0 <= b < cdf.size - 1 and cdf[b] - margin <= u[r, k] < cdf[b + 1] + margin
                bad += int(not ok)
    return bad, near


def grad_blocks(a, g, want):
    """Cosine and relative L2 error of a gradient against the oracle's, per hash
    level and per MLP matrix (blocks the oracle leaves at zero are skipped), so
    that an error in a block of small entries is not hidden by the large ones."""
    g = np.asarray(g, np.float64)
    want = np.asarray(want, np.float64)
    spans = [(f"level {l}", orc.level_offset(a, l), orc.level_offset(a, l + 1)) for l in range(a.L)]
    spans += [(f"layer {k}", orc.mlp_offset(a, k), orc.mlp_offset(a, k + 1)) for k in range(a.hidden + 1)]
    out = {}
    for name, lo, hi in spans:
        x, y = g[lo:hi], want[lo:hi]
        ny = np.linalg.norm(y)
        if ny == 0.0:
            continue
        nx = np.linalg.norm(x)
        out[name] = (float(x @ y / (nx * ny)) if nx > 0 else 0.0, float(np.linalg.norm(x - y) / ny))
    return out


def worst_blocks(a, g, want):
    """(smallest cosine, largest relative L2, the blocks they come from) over grad_blocks."""
    b = grad_blocks(a, g, want)
    kc = min(b, key=lambda k: b[k][0])
    kl = max(b, key=lambda k: b[k][1])
    return b[kc][0], b[kl][1], (kc, kl)
