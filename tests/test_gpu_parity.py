"""CUDA path against the FP64 oracle, element by element, on seeded synthetic scenes.

Acceptance (per tensor, max |gpu - oracle| / max |oracle|): forward outputs
(colour, depth, opacity, loss) <= 1e-5, gradients <= 1e-4; sample bins exact
away from CDF edges (1e-5 margin, either neighbour inside it).
"""

import numpy as np
import pytest

from helpers import CFG1, CFG2, bins_match, case, conditioned_uniforms, oracle_samples, oracle_t, rel

import oracle as orc

pytestmark = pytest.mark.gpu

FWD_TOL = 1e-5
GRAD_TOL = 1e-4


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_01582_gb300 import build

    build.build()
    import paper_2503_01582_gb300 as p

    return p


def _arch(p, d):
    return p.make_arch(L=d["L"], F=d["F"], log2T=d["log2T"], n_min=d["n_min"], n_max=d["n_max"], width=d["width"],
                       hidden=d["hidden"], lambda_d=d["lambda_d"], lambda_sigma=d["lambda_sigma"])


def _dev(rays, obj, u=None, cr=None, t_in=None):
    import torch

    b = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.items()}
    b["obj"] = obj
    if u is not None:
        b["uniforms"] = torch.from_numpy(np.ascontiguousarray(u, dtype=np.float32)).cuda()
    if cr is not None:
        b["c_rand"] = torch.from_numpy(np.ascontiguousarray(cr, dtype=np.float32)).cuda()
    if t_in is not None:
        b["t_in"] = torch.from_numpy(np.ascontiguousarray(t_in, dtype=np.float32)).cuda()
    return b


def _setup(pkg, arch, theta, grid):
    ctx = pkg.Context(seed=7)
    obj = ctx.create_object(_arch(pkg, arch), theta)
    ctx.set_prior_grid(obj, grid)
    return ctx, obj


def test_layout_contract(pkg):
    for arch in (CFG1, CFG2, dict(CFG1, L=4, log2T=12, n_max=32, width=16, hidden=3)):
        a = orc.Arch(**arch)
        ctx = pkg.Context()
        obj = ctx.create_object(_arch(pkg, arch))
        assert ctx.param_count(obj) == orc.param_count(a)
        res, off, dense = ctx.level_info(obj)
        assert res == [orc.level_res(a, l) for l in range(a.L)]
        assert off == [orc.level_offset(a, l) for l in range(a.L + 1)]
        assert dense == [orc.level_dense(a, l) for l in range(a.L)]
        ctx.close()


@pytest.mark.parametrize("nc,nr", [(32, 32), (64, 64), (48, 48), (7, 5)])
def test_sampler_bins_and_depths(pkg, nc, nr):
    a, theta, grid, rays, u, cr = case(CFG1, 300, nr, nc, seed=3)
    ctx, obj = _setup(pkg, CFG1, theta, grid)
    opts = pkg.make_opts(nc=nc, nr=nr)
    out = ctx.render(_dev(rays, obj, u), opts, want_samples=True)
    gb = out["bins"].cpu().numpy()
    gt = out["t"].cpu().numpy().astype(np.float64)
    want = oracle_samples(grid, rays, u, nc, nr)
    bad, near = bins_match(gb, want["bins"], want["cdf"], u)
    assert bad == 0, (bad, near)
    assert near <= 0.001 * u.size + 2
    # depths: the FP32 CDF error (a few 1e-7) is divided by the bin mass
    delta = (want["tf"] - want["tn"]) / nc
    mass = np.take_along_axis(np.diff(want["cdf"], axis=1), want["bins"], axis=1)
    tol = delta[:, None] * 2e-6 / np.maximum(mass, 1e-30) + 1e-6 * np.abs(want["t"]) + 1e-7
    ok = (gb == want["bins"])
    assert np.all(np.abs(gt - want["t"])[ok] <= tol[ok])
    ctx.close()


def test_sampler_special_cases(pkg):
    import torch

    R = 16
    o = np.array([[-1.0, 0.5, 0.5], [-1.0, 0.31, 0.52], [0.5, 0.5, 0.5]], np.float32)
    d = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]], np.float32)
    rays = dict(o=o, d=d)
    nc, nr = 32, 32
    u = np.sort(np.random.default_rng(0).random((3, nr)).astype(np.float32), axis=1)
    a = orc.Arch(**CFG1)
    theta = np.zeros(orc.param_count(a), np.float32)
    for name, grid in [("escape", np.zeros((R, R, R), np.float32)),
                       ("one-hot", np.where(np.arange(R)[None, None, :] >= 10, 1e30, 0.0).repeat(R, 0).repeat(R, 1)
                        .astype(np.float32)),
                       ("constant", np.full((R, R, R), 3.0, np.float32))]:
        grid = np.ascontiguousarray(np.broadcast_to(grid, (R, R, R)), dtype=np.float32)
        ctx, obj = _setup(pkg, CFG1, theta, grid)
        out = ctx.render(_dev(rays, obj, u), pkg.make_opts(nc=nc, nr=nr), want_samples=True)
        gb = out["bins"].cpu().numpy()
        want = oracle_samples(grid, rays, u, nc, nr)
        bad, near = bins_match(gb, want["bins"], want["cdf"], u)
        assert bad == 0, name
        if name == "escape":
            assert want["escape"].all()
            np.testing.assert_array_equal(gb, np.floor(u * nc).astype(np.int32))
        if name == "one-hot":
            assert np.all(gb[0] == gb[0, 0]) and np.all(gb[1] == gb[1, 0])
        ctx.close()
    torch.cuda.synchronize()


def test_forward_given_samples(pkg):
    """Encoding, MLP, compositing on the oracle's own sample depths (rounded to FP32)."""
    a, theta, grid, rays, u, cr = case(CFG1, 256, 32, 32, seed=5, hash_range=0.5)
    want_s = oracle_samples(grid, rays, u, 32, 32)
    t_in = want_s["t"].astype(np.float32)
    want = orc.batch(a, theta, grid, rays, 32, 32, t_in=t_in, c_rand=cr)
    ctx, obj = _setup(pkg, CFG1, theta, grid)
    out = ctx.render(_dev(rays, obj, t_in=t_in), pkg.make_opts(nc=32, nr=32), want_samples=True)
    np.testing.assert_array_equal(out["t"].cpu().numpy(), t_in)
    for k in ("rgb", "depth", "acc"):
        e = rel(out[k].cpu().numpy(), want[k])
        assert e <= FWD_TOL, (k, e)
    ctx.close()


ARCHS = [CFG1, dict(CFG1, lambda_sigma=1e-2), dict(CFG1, L=4, log2T=12, n_max=64, width=16, hidden=3),
         dict(CFG1, L=16, log2T=15, n_max=512, width=64, hidden=1)]


def _check_grads(a, g, want, exact_zeros=True):
    nh = orc.n_hash_params(a)
    for l in range(a.L):
        lo, hi = orc.level_offset(a, l), orc.level_offset(a, l + 1)
        assert rel(g[lo:hi], want[lo:hi]) <= GRAD_TOL, ("level", l, rel(g[lo:hi], want[lo:hi]))
    for layer in range(a.hidden + 1):
        lo, hi = orc.mlp_offset(a, layer), orc.mlp_offset(a, layer + 1)
        assert rel(g[lo:hi], want[lo:hi]) <= GRAD_TOL, ("layer", layer, rel(g[lo:hi], want[lo:hi]))
    if exact_zeros:  # on identical samples, entries no sample touches stay exactly zero
        assert np.all(g[:nh][want[:nh] == 0] == 0)


@pytest.mark.parametrize("arch", ARCHS)
def test_loss_and_gradients_on_identical_samples(pkg, arch):
    import torch

    a, theta, grid, rays, u, cr = case(arch, 200, 32, 32, seed=11, hash_range=0.5)
    t_in = oracle_t(grid, rays, u, 32, 32)
    want = orc.batch(a, theta, grid, rays, 32, 32, t_in=t_in, c_rand=cr, want_grad=True)
    ctx, obj = _setup(pkg, arch, theta, grid)
    b = _dev(rays, obj, cr=cr, t_in=t_in)
    out = ctx.render(b, pkg.make_opts(nc=32, nr=32))
    for k in ("rgb", "depth", "acc"):
        assert rel(out[k].cpu().numpy(), want[k]) <= FWD_TOL, k
    loss = torch.zeros(1, device="cuda")
    ctx.train_step([b], pkg.make_opts(nc=32, nr=32, flags=pkg.PRENOM_FLAG_NO_ADAM), loss)
    assert abs(loss.item() - want["loss"]) <= FWD_TOL * abs(want["loss"])
    _check_grads(a, ctx.get_state(obj, pkg.PRENOM_STATE_GRAD).cpu().numpy(), want["grad"])
    ctx.close()


@pytest.mark.parametrize("nr", [80, 96, 128])
def test_long_rays_over_several_warps(pkg, nr):
    """Rays of more than 64 samples: the compositing spreads each over
    ceil(nr/32) = 3 or 4 warps (the last one partly filled for nr = 80), which
    meet through named barriers; a tile holds one such ray.  Forward, loss and
    gradients on identical samples against the oracle, both forms."""
    import torch

    a, theta, grid, rays, u, cr = case(CFG1, 37, nr, 32, seed=61, hash_range=0.5)
    t_in = oracle_t(grid, rays, u, 32, nr)
    want = orc.batch(a, theta, grid, rays, 32, nr, t_in=t_in, c_rand=cr, want_grad=True)
    for flags in (0, pkg.PRENOM_FLAG_FUSED):
        ctx, obj = _setup(pkg, CFG1, theta, grid)
        b = _dev(rays, obj, cr=cr, t_in=t_in)
        out = ctx.render(b, pkg.make_opts(nc=32, nr=nr))
        for k in ("rgb", "depth", "acc"):
            assert rel(out[k].cpu().numpy(), want[k]) <= FWD_TOL, (k, flags)
        loss = torch.zeros(1, device="cuda")
        ctx.train_step([b], pkg.make_opts(nc=32, nr=nr, flags=flags | pkg.PRENOM_FLAG_NO_ADAM), loss)
        assert abs(loss.item() - want["loss"]) <= FWD_TOL * abs(want["loss"]), flags
        _check_grads(a, ctx.get_state(obj, pkg.PRENOM_STATE_GRAD).cpu().numpy(), want["grad"])
        ctx.close()


@pytest.mark.parametrize("arch", ARCHS[:2])
def test_end_to_end_from_uniforms(pkg, arch):
    """Sampler included: uniforms kept out of bins lighter than 2 % of the ray's mass."""
    import torch

    a, theta, grid, rays, _, cr = case(arch, 200, 32, 32, seed=13, hash_range=0.5)
    u = conditioned_uniforms(grid, rays, 32, 32, seed=14)
    want = orc.batch(a, theta, grid, rays, 32, 32, u=u, c_rand=cr, want_grad=True)
    ctx, obj = _setup(pkg, arch, theta, grid)
    b = _dev(rays, obj, u, cr)
    out = ctx.render(b, pkg.make_opts(nc=32, nr=32))
    for k in ("rgb", "depth", "acc"):
        assert rel(out[k].cpu().numpy(), want[k]) <= FWD_TOL, k
    loss = torch.zeros(1, device="cuda")
    ctx.train_step([b], pkg.make_opts(nc=32, nr=32, flags=pkg.PRENOM_FLAG_NO_ADAM), loss)
    assert abs(loss.item() - want["loss"]) <= FWD_TOL * abs(want["loss"])
    # a sample depth that differs in the last bits may put a zero-weight corner in
    # the neighbouring cell, so only the values (not the support) must agree here
    _check_grads(a, ctx.get_state(obj, pkg.PRENOM_STATE_GRAD).cpu().numpy(), want["grad"], exact_zeros=False)
    ctx.close()


def test_adam_one_step_and_trajectory(pkg):
    import torch

    a, theta, grid, rays0, u0, cr0 = case(CFG1, 256, 32, 32, seed=21)
    ob = orc.OracleObject(a, theta, grid)
    ctx, obj = _setup(pkg, CFG1, theta, grid)
    from helpers import pool_cfg1
    from synth import random_colours, sample_batch, stratified_uniforms

    _, pool = pool_cfg1()
    losses_g, losses_o = [], []
    loss = torch.zeros(1, device="cuda")
    for step in range(20):
        rays = sample_batch(pool, 256, 100 + step)
        u = stratified_uniforms(256, 32, 200 + step)
        cr = random_colours(256, 300 + step)
        t_in = oracle_t(grid, rays, u, 32, 32)  # the samples do not depend on theta
        losses_o.append(ob.train_step(rays, 32, 32, t_in=t_in, c_rand=cr, lr=1e-2))
        ctx.train_step([_dev(rays, obj, cr=cr, t_in=t_in)], pkg.make_opts(nc=32, nr=32, lr=1e-2), loss)
        losses_g.append(loss.item())
        if step == 0:
            th = ctx.get_state(obj, pkg.PRENOM_STATE_THETA).cpu().numpy()
            g_o = orc.batch(a, theta, grid, rays, 32, 32, t_in=t_in, c_rand=cr, want_grad=True)["grad"]
            # Adam normalises each gradient entry: where the oracle gradient is
            # below the FP32 noise floor the sign of the first step is arbitrary
            sure = np.abs(g_o) > 1e-5 * np.abs(g_o).max()
            d = np.abs(th - ob.theta)
            assert np.max(d[sure]) <= GRAD_TOL * np.abs(ob.theta).max()
            assert np.max(d[~sure], initial=0.0) <= 2.01e-2
    lg, lo = np.array(losses_g), np.array(losses_o)
    assert np.all(np.abs(lg - lo) <= GRAD_TOL * np.abs(lo)), np.abs(lg - lo) / np.abs(lo)
    assert ctx.get_step(obj) == 20
    ctx.close()


def test_edge_cases(pkg):
    import torch

    a, theta, grid, rays, u, cr = case(CFG1, 37, 48, 16, seed=31)
    ctx, obj = _setup(pkg, CFG1, theta, grid)
    opts = pkg.make_opts(nc=16, nr=48, flags=pkg.PRENOM_FLAG_NO_ADAM)
    # empty batch: no work, loss 0
    loss = torch.ones(1, device="cuda")
    empty = {k: v[:0] for k, v in _dev(rays, obj, u, cr).items() if k != "obj"}
    empty["obj"] = obj
    ctx.train_step([empty], opts, loss)
    assert loss.item() == 0.0
    # ragged: 37 rays of 48 samples (2 rays per 128-sample tile, 1 in the last)
    t_in = oracle_t(grid, rays, u, 16, 48)
    want = orc.batch(a, theta, grid, rays, 16, 48, t_in=t_in, c_rand=cr, want_grad=True)
    ctx.train_step([_dev(rays, obj, cr=cr, t_in=t_in)], opts, loss)
    assert abs(loss.item() - want["loss"]) <= FWD_TOL * abs(want["loss"])
    g = ctx.get_state(obj, pkg.PRENOM_STATE_GRAD).cpu().numpy()
    assert rel(g, want["grad"]) <= GRAD_TOL
    # rays that miss the cube and rays starting inside it
    miss = dict(o=np.array([[-1, 2, 0.5], [0.5, 0.5, 0.5], [0.2, 0.9, 0.1]], np.float32),
                d=np.array([[1, 0, 0], [0, 0.6, 0.8], [0.6, -0.8, 0.0]], np.float32),
                rgb=np.full((3, 3), 0.5, np.float32), depth=np.ones(3, np.float32),
                is_obj=np.array([1, 1, 0], np.uint8))
    um = u[:3]
    want = orc.batch(a, theta, grid, miss, 16, 48, u=um, c_rand=cr[:3])
    out = ctx.render(_dev(miss, obj, um, cr[:3]), opts)
    for k in ("rgb", "depth", "acc"):
        assert rel(out[k].cpu().numpy(), want[k]) <= FWD_TOL, k
    assert out["acc"][0].item() == 0.0
    ctx.close()


def test_render_backward_matches_oracle(pkg):
    import torch

    a, theta, grid, rays, u, cr = case(CFG1, 128, 32, 32, seed=41, hash_range=0.5)
    up = np.random.default_rng(1).normal(size=(128, 5))
    t_in = oracle_t(grid, rays, u, 32, 32)
    want = orc.batch(a, theta, grid, rays, 32, 32, t_in=t_in, upstream=up.astype(np.float32), want_grad=True)
    ctx, obj = _setup(pkg, CFG1, theta, grid)
    grad = torch.zeros(ctx.param_count(obj), device="cuda")
    ctx.render_backward(_dev(rays, obj, t_in=t_in), pkg.make_opts(nc=32, nr=32),
                        torch.from_numpy(up.astype(np.float32)).cuda(), grad)
    assert rel(grad.cpu().numpy(), want["grad"]) <= GRAD_TOL
    # through torch.autograd
    from paper_2503_01582_gb300.autograd import render

    th = torch.from_numpy(theta).cuda().requires_grad_(True)
    rgb, depth, acc = render(ctx, obj, th, _dev(rays, obj, t_in=t_in), pkg.make_opts(nc=32, nr=32))
    upt = torch.from_numpy(up.astype(np.float32)).cuda()
    (rgb * upt[:, :3]).sum().add((depth * upt[:, 3]).sum()).add((acc * upt[:, 4]).sum()).backward()
    assert rel(th.grad.cpu().numpy(), want["grad"]) <= GRAD_TOL
    ctx.close()


def test_autograd_render_matches_central_differences(pkg):
    """The GPU backward through torch.autograd against central differences of
    the GPU forward itself (FP32), on the L = 4, T = 2^12 architecture: for the
    hash entries and MLP weights with the largest gradients, (f(theta + h e_i) -
    f(theta - h e_i)) / 2h with h = 1e-2 max(|theta_i|, 0.1) agrees with the
    analytic gradient to 1e-2.  Entries are kept only where the oracle's own
    central difference at the same points (FP64) matches the oracle's analytic
    gradient to 2e-3, so that the step h does not cross a ReLU or cell kink."""
    import torch

    from paper_2503_01582_gb300.autograd import render

    arch = dict(L=4, F=2, log2T=12, n_min=4, n_max=32, width=16, hidden=2, lambda_d=0.1, lambda_sigma=0.0)
    a, theta, grid, rays, u, cr = case(arch, 32, 16, 16, seed=101, hash_range=0.5)
    t_in = oracle_t(grid, rays, u, 16, 16)
    up = np.random.default_rng(7).normal(size=(32, 5)).astype(np.float32)
    ctx, obj = _setup(pkg, arch, theta, grid)
    batch = _dev(rays, obj, t_in=t_in)
    opts = pkg.make_opts(nc=16, nr=16)
    upt = torch.from_numpy(up).cuda()

    def f_gpu(th):
        rgb, depth, acc = render(ctx, obj, th, batch, opts)
        return (rgb * upt[:, :3]).sum() + (depth * upt[:, 3]).sum() + (acc * upt[:, 4]).sum()

    th = torch.from_numpy(theta.astype(np.float32)).cuda().requires_grad_(True)
    f_gpu(th).backward()
    g = th.grad.cpu().numpy().astype(np.float64)

    def f_orc(tt):
        return orc.batch(a, tt, grid, rays, 16, 16, t_in=t_in, upstream=up, want_samples=False)["loss"]

    g64 = orc.batch(a, theta.astype(np.float64), grid, rays, 16, 16, t_in=t_in, upstream=up, want_grad=True)["grad"]
    nh = orc.n_hash_params(a)
    cand = np.concatenate([np.argsort(-np.abs(g64[:nh]))[:40], nh + np.argsort(-np.abs(g64[nh:]))[:40]])
    kept, bad = 0, []
    th0 = theta.astype(np.float32)
    with torch.no_grad():
        for i in cand:
            h = np.float32(1e-2 * max(abs(float(th0[i])), 0.1))
            hi, lo = th0.copy(), th0.copy()
            hi[i] = th0[i] + h
            lo[i] = th0[i] - h
            den = float(hi[i]) - float(lo[i])  # the FP32 points both sides evaluate
            fd64 = (f_orc(hi.astype(np.float64)) - f_orc(lo.astype(np.float64))) / den
            if abs(fd64 - g64[i]) > 2e-3 * abs(g64[i]):
                continue  # a kink inside [theta_i - h, theta_i + h]
            kept += 1
            fd = (float(f_gpu(torch.from_numpy(hi).cuda())) - float(f_gpu(torch.from_numpy(lo).cuda()))) / den
            if abs(fd - g[i]) > 1e-2 * abs(g[i]) + 1e-6 * np.abs(g).max():
                bad.append((int(i), fd, g[i]))
    assert kept >= 40, kept
    assert not bad, bad
    ctx.close()


def test_philox_draws_match_oracle(pkg):
    import torch

    a, theta, grid, rays, u, cr = case(CFG1, 96, 32, 32, seed=51)
    ctx = pkg.Context(seed=0x1234567890AB)
    obj = ctx.create_object(_arch(pkg, CFG1), theta)
    ctx.set_prior_grid(obj, grid)
    ctx.set_step(obj, 5)
    out = ctx.render(_dev(rays, obj), pkg.make_opts(nc=32, nr=32), want_samples=True)
    uu = orc.philox_uniforms(0x1234567890AB, 5, obj, 96, 32)
    want = oracle_samples(grid, rays, uu, 32, 32)
    bad, _ = bins_match(out["bins"].cpu().numpy(), want["bins"], want["cdf"], uu)
    assert bad == 0
    crr = orc.philox_colours(0x1234567890AB, 5, obj, 96)
    w = orc.batch(a, theta, grid, rays, 32, 32, u=uu, c_rand=crr)
    loss = torch.zeros(1, device="cuda")
    ctx.train_step([_dev(rays, obj)], pkg.make_opts(nc=32, nr=32, flags=pkg.PRENOM_FLAG_NO_ADAM), loss)
    assert abs(loss.item() - w["loss"]) <= FWD_TOL * abs(w["loss"])
    ctx.close()


def test_random_init_and_errors(pkg):
    import torch

    ctx = pkg.Context(seed=3)
    obj = ctx.create_object(_arch(pkg, CFG1))
    th = ctx.get_state(obj).cpu().numpy()
    a = orc.Arch(**CFG1)
    nh = orc.n_hash_params(a)
    assert np.abs(th[:nh]).max() <= 1e-4 and np.abs(th[:nh]).max() > 0.9e-4
    assert abs(th[:nh].mean()) < 1e-6
    lim = np.sqrt(6.0 / (16 + 32))
    w1 = th[nh:nh + 32 * 16]
    assert np.abs(w1).max() <= lim and np.abs(w1).max() > 0.9 * lim
    with pytest.raises(pkg.PrenomError) as e:
        ctx.create_object(_arch(pkg, dict(CFG1, width=48)))
    assert e.value.code == -1
    with pytest.raises(pkg.PrenomError) as e:  # no prior grid
        ctx.render(dict(obj=obj, o=torch.zeros((4, 3), device="cuda"), d=torch.ones((4, 3), device="cuda")),
                   pkg.make_opts())
    assert e.value.code == -1
    with pytest.raises(pkg.PrenomError):
        ctx.train_step([dict(obj=99, o=torch.zeros((4, 3), device="cuda"), d=torch.ones((4, 3), device="cuda"))],
                       pkg.make_opts())
    with pytest.raises(pkg.PrenomError):
        ctx.render(dict(obj=obj, o=torch.zeros((4, 3), device="cuda"), d=torch.ones((4, 3), device="cuda")),
                   pkg.make_opts(nr=200))
    ctx.close()


def test_full_size_config_sampled(pkg):
    """The 16-level, 2^19-entry, 2x64 MLP object at 4096 rays x 64 samples in the
    launch configuration the benchmark times: the oracle checks the outputs of
    sampled rays of the full batch (from uniforms), and the loss and every
    gradient of a 64-ray batch of the same object on identical samples."""
    import torch

    arch = CFG2
    a = orc.Arch(**arch)
    from helpers import pool_cfg2
    from synth import init_params, prior_grid, random_colours, sample_batch, stratified_uniforms

    sc, pool = pool_cfg2()
    rays = sample_batch(pool, 4096, 0)
    u = stratified_uniforms(4096, 64, 1)
    cr = random_colours(4096, 2)
    grid = prior_grid(sc, 64, 0)
    theta = init_params(orc.n_hash_params(a), a.mlp_shapes(), 3, hash_range=0.5)
    ctx, obj = _setup(pkg, arch, theta, grid)
    idx = np.random.default_rng(0).choice(4096, 48, replace=False)
    sub = {k: v[idx] for k, v in rays.items()}
    # the sampler over the whole batch: bins of the sampled rays exact outside the edge margin
    out = ctx.render(_dev(rays, obj, u, cr), pkg.make_opts(nc=64, nr=64), want_samples=True)
    ws = oracle_samples(grid, sub, u[idx], 64, 64)
    bad, _ = bins_match(out["bins"].cpu().numpy()[idx], ws["bins"], ws["cdf"], u[idx])
    assert bad == 0
    # field and rendering over the whole batch on identical samples: at the finest
    # level (n_max 2048) one FP32 ulp of t already moves a feature by ~1e-5
    t_all = oracle_t(grid, rays, u, 64, 64)
    out = ctx.render(_dev(rays, obj, cr=cr, t_in=t_all), pkg.make_opts(nc=64, nr=64))
    want = orc.batch(a, theta, grid, sub, 64, 64, t_in=t_all[idx], c_rand=cr[idx])
    for k in ("rgb", "depth", "acc"):
        assert rel(out[k].cpu().numpy()[idx], want[k]) <= FWD_TOL, k
    # gradients of a 64-ray batch at full architecture size
    sub = {k: v[:64] for k, v in rays.items()}
    t_in = oracle_t(grid, sub, u[:64], 64, 64)
    want = orc.batch(a, theta, grid, sub, 64, 64, t_in=t_in, c_rand=cr[:64], want_grad=True)
    loss = torch.zeros(1, device="cuda")
    ctx.train_step([_dev(sub, obj, cr=cr[:64], t_in=t_in)],
                   pkg.make_opts(nc=64, nr=64, flags=pkg.PRENOM_FLAG_NO_ADAM), loss)
    assert abs(loss.item() - want["loss"]) <= FWD_TOL * abs(want["loss"])
    g = ctx.get_state(obj, pkg.PRENOM_STATE_GRAD).cpu().numpy()
    _check_grads(a, g, want["grad"])  # per level and per layer
    ctx.close()
