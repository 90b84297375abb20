"""Prior density grid from the field (§III-A, §III-B refresh) and the yaw
canonicalisation of Eq. 3 on the GPU against the FP64 oracle."""

import numpy as np
import pytest

from helpers import CFG1, CFG2, rel

import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_01582_gb300 import build

    build.build()
    import paper_2503_01582_gb300 as p

    return p


def _arch(p, d, precision=0):
    return p.make_arch(L=d["L"], F=d["F"], log2T=d["log2T"], n_min=d["n_min"], n_max=d["n_max"], width=d["width"],
                       hidden=d["hidden"], lambda_d=d["lambda_d"], lambda_sigma=d["lambda_sigma"], precision=precision)


@pytest.mark.parametrize("arch,res", [(CFG1, 32), (CFG1, 64), (CFG2, 64), (dict(CFG1, width=64, hidden=3), 64)])
def test_density_grid_against_oracle(pkg, arch, res):
    from synth import init_params

    a = orc.Arch(**arch)
    theta = init_params(orc.n_hash_params(a), a.mlp_shapes(), 7, hash_range=0.5).astype(np.float32)
    ctx = pkg.Context(seed=1)
    obj = ctx.create_object(_arch(pkg, arch), theta)
    g = ctx.density_grid(obj, res).cpu().numpy()
    want = orc.density_grid(a, theta, res)
    # voxel centres of a power-of-two grid are exact in FP32: only the FP32 forward differs
    assert rel(g, want) <= 1e-5, rel(g, want)
    assert np.all(np.isfinite(g)) and np.all(g > 0)
    ctx.close()


@pytest.mark.parametrize("precision,bound", [(1, 5e-3), (2, 3e-2)])
def test_density_grid_mixed_precision(pkg, precision, bound):
    from synth import init_params

    a = orc.Arch(**CFG1)
    theta = init_params(orc.n_hash_params(a), a.mlp_shapes(), 8, hash_range=0.5).astype(np.float32)
    ctx = pkg.Context(seed=1)
    obj = ctx.create_object(_arch(pkg, CFG1, precision), theta)
    g = ctx.density_grid(obj, 32).cpu().numpy()
    want = orc.density_grid(a, theta, 32)
    # sigma = exp(o_0): the 16-bit MLP's absolute output error becomes a relative density error
    assert np.max(np.abs(g / want - 1)) <= bound
    ctx.close()


def test_refresh_prior_then_sampling_uses_it(pkg):
    """After a refresh the object's prior grid is its own density: the sampler's
    bins follow the oracle's on that grid."""
    import torch
    from helpers import bins_match, case, oracle_samples

    a, theta, grid, rays, u, cr = case(CFG1, 64, 32, 32, seed=4, hash_range=0.5)
    ctx = pkg.Context(seed=1)
    obj = ctx.create_object(_arch(pkg, CFG1), theta)
    ctx.set_prior_grid(obj, grid)
    ctx.refresh_prior(obj, 32)
    new_grid = orc.density_grid(a, theta, 32)
    b = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.items()}
    b["obj"] = obj
    b["uniforms"] = torch.from_numpy(u).cuda()
    out = ctx.render(b, pkg.make_opts(nc=32, nr=32), want_samples=True)
    gpu_grid = ctx.density_grid(obj, 32).cpu().numpy()
    ws = oracle_samples(gpu_grid.astype(np.float64), rays, u, 32, 32)
    bad, _ = bins_match(out["bins"].cpu().numpy(), ws["bins"], ws["cdf"], u)
    assert bad == 0
    assert rel(gpu_grid, new_grid) <= 1e-5
    ctx.close()


def _l_shape(n, seed):
    rng = np.random.default_rng(seed)
    a = np.c_[rng.uniform(-0.5, 0.5, n // 2), rng.uniform(-0.5, -0.3, n // 2)]
    b = np.c_[rng.uniform(-0.5, -0.3, n // 2), rng.uniform(-0.3, 0.2, n // 2)]
    xy = np.r_[a, b]
    return np.c_[xy, rng.uniform(-0.2, 0.2, xy.shape[0])]


def _splat(P, R):
    lo, hi = P.min(0), P.max(0)
    Pn = (P - 0.5 * (lo + hi)) / (hi - lo) + 0.5
    g = np.zeros((R, R, R))
    idx = np.clip((Pn * R).astype(int), 0, R - 1)
    np.add.at(g, (idx[:, 2], idx[:, 1], idx[:, 0]), 1.0)
    return g


@pytest.mark.parametrize("n_points,n_gamma", [(1000, 36), (20000, 360), (5, 8)])
def test_canonical_yaw_against_oracle(pkg, n_points, n_gamma):
    import torch

    P = _l_shape(max(n_points, 2), 1)[:n_points]
    grid = _splat(_l_shape(4000, 2), 32)
    ctx = pkg.Context(seed=1)
    obj = ctx.create_object(_arch(pkg, CFG1))
    ctx.set_prior_grid(obj, grid.astype(np.float32))
    for g0 in (0, n_gamma // 3, n_gamma - 1):
        ang = -2 * np.pi * g0 / n_gamma
        c, s = np.cos(ang), np.sin(ang)
        Q = (P @ np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]]).T).astype(np.float32)
        best, scores = ctx.canonical_yaw(obj, torch.from_numpy(Q).cuda(), n_gamma)
        want_best, want = orc.canonical_yaw(grid.astype(np.float32), Q, n_gamma)
        sc = scores.cpu().numpy()
        assert rel(sc, want) <= 1e-5
        # the argmax is unique up to the scores' precision: the GPU's choice scores like the oracle's best
        assert want[best] >= want[want_best] * (1 - 1e-5)
        if n_points >= 1000:
            assert best == want_best == g0
    ctx.close()
