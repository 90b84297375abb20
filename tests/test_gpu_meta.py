"""Reptile meta step (§III-A, Eq. 1-2) on the GPU against the FP64 oracle."""

import numpy as np
import pytest

from helpers import CFG1, case, oracle_t, rel

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


def _dev(rays, obj, cr=None, t_in=None):
    import torch

    b = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.items()}
    b["obj"] = obj
    if cr is not None:
        b["c_rand"] = torch.from_numpy(np.ascontiguousarray(cr, dtype=np.float32)).cuda()
    if t_in is not None:
        b["t_in"] = torch.from_numpy(np.ascontiguousarray(t_in, dtype=np.float32)).cuda()
    return b


@pytest.mark.parametrize("n_tasks", [1, 3, 16])
def test_begin_and_outer_update_against_oracle(pkg, n_tasks):
    import torch

    a = orc.Arch(**CFG1)
    n = orc.param_count(a)
    rng = np.random.default_rng(n_tasks)
    ctx = pkg.Context(seed=1)
    meta = ctx.create_object(_arch(pkg, CFG1), rng.normal(size=n).astype(np.float32))
    tasks = [ctx.create_object(_arch(pkg, CFG1, precision=t % 2)) for t in range(n_tasks)]
    ctx.set_state(tasks[0], pkg.PRENOM_STATE_ADAM_M, torch.ones(n, device="cuda"))
    ctx.set_step(tasks[0], 7)
    ctx.reptile_begin(meta, tasks)
    th_meta = ctx.get_state(meta).cpu().numpy()
    for t in tasks:
        np.testing.assert_array_equal(ctx.get_state(t).cpu().numpy(), th_meta)
        for which in (pkg.PRENOM_STATE_GRAD, pkg.PRENOM_STATE_ADAM_M, pkg.PRENOM_STATE_ADAM_V):
            assert not ctx.get_state(t, which).cpu().numpy().any()
        assert ctx.get_step(t) == 0
    # arbitrary task results, then Eq. 2 over the meta-batch
    finals = [rng.normal(size=n).astype(np.float32) for _ in tasks]
    for t, f in zip(tasks, finals):
        ctx.set_state(t, pkg.PRENOM_STATE_THETA, torch.from_numpy(f).cuda())
    want = th_meta.astype(np.float64)
    orc.reptile(want, finals, 0.3)
    ctx.reptile_update(meta, tasks, 0.3)
    got = ctx.get_state(meta).cpu().numpy()
    assert rel(got, want) <= 1e-6
    # the two-call form (task sum, then apply) computes the same update
    meta2 = ctx.create_object(_arch(pkg, CFG1), th_meta)
    s = torch.empty(n, device="cuda")
    ctx.reptile_task_sum(tasks, s)
    np.testing.assert_allclose(s.cpu().numpy(), np.sum(np.array(finals, np.float64), axis=0), rtol=1e-6, atol=1e-5)
    ctx.reptile_apply(meta2, s, n_tasks, 0.3)
    np.testing.assert_array_equal(ctx.get_state(meta2).cpu().numpy(), got)
    # errors: duplicate task, meta among tasks, another architecture, beta out of range
    other = ctx.create_object(_arch(pkg, dict(CFG1, width=16)))
    for bad in ([tasks[0], tasks[0]], [meta], [other]):
        with pytest.raises(pkg.PrenomError):
            ctx.reptile_update(meta, bad, 0.3)
    with pytest.raises(pkg.PrenomError):
        ctx.reptile_update(meta, tasks, 1.5)
    ctx.close()


def test_meta_step_against_oracle(pkg):
    """A whole meta step: 3 tasks (one CSG topology, per-task scale jitter), 3
    inner Adam steps each on identical samples, then Eq. 2 with beta = 0.1; the
    inner losses and the new meta-parameters match the oracle's meta step."""
    import torch
    from helpers import CFG1 as A
    from paper_2503_01582_gb300.meta import meta_step
    from synth import (cameras_on_sphere, init_params, make_ray_pool, prior_grid, random_colours, sample_batch,
                       scene_random_csg, stratified_uniforms)

    a = orc.Arch(**A)
    theta0 = init_params(orc.n_hash_params(a), a.mlp_shapes(), 11, hash_range=0.5).astype(np.float32)
    scales = [0.85, 1.0, 1.15]
    grids, pools = [], []
    for i, sc_ in enumerate(scales):
        sc = scene_random_csg(5, scale=sc_)
        grids.append(prior_grid(sc, 32, i))
        pools.append(make_ray_pool(sc, cameras_on_sphere(8, 2.0, 40, 64, 64, i), 4096, i))
    q = 3
    host = [[] for _ in scales]  # per task, per inner step: rays + identical samples
    for t in range(len(scales)):
        for j in range(q):
            rays = sample_batch(pools[t], 128, 100 * t + j)
            u = stratified_uniforms(128, 32, 200 * t + j)
            host[t].append(dict(rays, t_in=oracle_t(grids[t], rays, u, 32, 32), c_rand=random_colours(128, 300 * t + j)))
    want, want_losses = orc.meta_step(a, theta0, lambda t: grids[t], host, 32, 32, lr=1e-2, beta=0.1)

    ctx = pkg.Context(seed=2)
    meta = ctx.create_object(_arch(pkg, A), theta0)
    tasks = [ctx.create_object(_arch(pkg, A)) for _ in scales]
    for t, g in zip(tasks, grids):
        ctx.set_prior_grid(t, g)
    inner = [[_dev({k: host[t][j][k] for k in ("o", "d", "rgb", "depth", "is_obj")}, tasks[t],
                   cr=host[t][j]["c_rand"], t_in=host[t][j]["t_in"]) for t in range(len(scales))] for j in range(q)]
    losses = torch.zeros(len(scales), device="cuda")
    got_losses = []

    class Recorder:  # records each inner step's losses through the same context
        def __getattr__(self, name):
            return getattr(ctx, name)

        def train_step(self, batches, opts, loss=None):
            ctx.train_step(batches, opts, losses)
            got_losses.append(losses.cpu().numpy().copy())

    n_total = meta_step(Recorder(), meta, tasks, inner, pkg.make_opts(nc=32, nr=32, lr=1e-2), 0.1)
    assert n_total == len(scales)
    got = ctx.get_state(meta).cpu().numpy()
    for j in range(q):
        for t in range(len(scales)):
            assert abs(got_losses[j][t] - want_losses[t][j]) <= 1e-4 * want_losses[t][j], (j, t)
    # Adam normalises each entry: compare the meta-parameters in bulk, and every
    # entry within the largest move the inner steps can make (beta x q x lr)
    diff = np.abs(got - want)
    assert np.mean(diff <= 1e-4 * np.abs(want).max() + 1e-7) > 0.999
    assert diff.max() <= 0.1 * q * 1e-2 * 1.01
    ctx.close()
