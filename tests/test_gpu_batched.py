"""Batched form: many objects with different tables, MLP widths and depths, ray
counts and precisions in one step, against the same objects stepped one at a
time (and, for the FP32 objects, against the FP64 oracle)."""

import numpy as np
import pytest

from helpers import CFG1, case, oracle_t, rel

import oracle as orc

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-4
FWD_TOL = 1e-5

# (log2T, width, hidden, L, precision, rays): a spread like a category table
OBJECTS = [(15, 32, 1, 16, 0, 160), (14, 32, 2, 8, 2, 96), (15, 64, 3, 16, 0, 200), (14, 64, 2, 16, 2, 130),
           (12, 16, 1, 8, 0, 64), (13, 32, 2, 16, 1, 256), (12, 16, 1, 4, 2, 72), (13, 16, 2, 8, 0, 100),
           (15, 64, 3, 8, 2, 180)]


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_01582_gb300 import build

    build.build()
    import paper_2503_01582_gb300 as p

    return p


def _setup(seed=0):
    objs = []
    for i, (log2T, W, H, L, prec, n) in enumerate(OBJECTS):
        arch = dict(CFG1, log2T=log2T, width=W, hidden=H, L=L, n_max=256 if L > 4 else 64)
        a, theta, grid, rays, u, cr = case(arch, n, 32, 32, seed=100 + 7 * i + seed, hash_range=0.5)
        t_in = oracle_t(grid, rays, u, 32, 32)
        objs.append(dict(arch=arch, prec=prec, a=a, theta=theta, grid=grid, rays=rays, cr=cr, t_in=t_in))
    return objs


def _batch(o, obj):
    import torch

    b = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in o["rays"].items()}
    b["obj"] = obj
    b["c_rand"] = torch.from_numpy(o["cr"]).cuda()
    b["t_in"] = torch.from_numpy(o["t_in"]).cuda()
    return b


def _make(pkg, objs, stream=None):
    ctx = pkg.Context(seed=1, stream=stream)
    ids = []
    for o in objs:
        ar = o["arch"]
        oid = ctx.create_object(pkg.make_arch(L=ar["L"], log2T=ar["log2T"], n_min=16, n_max=ar["n_max"],
                                              width=ar["width"], hidden=ar["hidden"], lambda_d=0.1,
                                              precision=o["prec"]), o["theta"])
        ctx.set_prior_grid(oid, o["grid"])
        ids.append(oid)
    return ctx, ids


def test_batched_gradients_match_per_object_and_oracle(pkg):
    import torch

    objs = _setup()
    opts = pkg.make_opts(nc=32, nr=32, flags=pkg.PRENOM_FLAG_NO_ADAM)
    ctx_b, ids_b = _make(pkg, objs)
    ctx_s, ids_s = _make(pkg, objs)
    loss_b = torch.zeros(len(objs), device="cuda")
    ctx_b.train_step([_batch(o, i) for o, i in zip(objs, ids_b)], opts, loss_b)
    for k, (o, i) in enumerate(zip(objs, ids_s)):
        loss_s = torch.zeros(1, device="cuda")
        ctx_s.train_step([_batch(o, i)], opts, loss_s)
        assert abs(loss_b[k].item() - loss_s.item()) <= FWD_TOL * abs(loss_s.item()), k
        gb = ctx_b.get_state(ids_b[k], pkg.PRENOM_STATE_GRAD).cpu().numpy()
        gs = ctx_s.get_state(i, pkg.PRENOM_STATE_GRAD).cpu().numpy()
        assert rel(gb, gs) <= GRAD_TOL, (k, rel(gb, gs))
        if o["prec"] == 0:
            want = orc.batch(o["a"], o["theta"], o["grid"], o["rays"], 32, 32, t_in=o["t_in"], c_rand=o["cr"],
                             want_grad=True)
            assert abs(loss_b[k].item() - want["loss"]) <= FWD_TOL * abs(want["loss"]), k
            assert rel(gb, want["grad"]) <= GRAD_TOL, (k, rel(gb, want["grad"]))
    ctx_b.close()
    ctx_s.close()


def test_batched_adam_graph_replay_and_autotuner(pkg):
    """Thirty-six batched steps on a side stream: the first nineteen tune the
    groups (one untimed call, then three rounds over the six candidates: the
    split form with two scatter variants and two encoder occupancies, the fused
    kernel with two work-chunk sizes), the next six time the whole step with its
    groups one after the other and forked onto side streams, the rest replay a
    captured graph while the ray buffers change.  Every step is checked against
    the same objects stepped one at a time (with PRENOM_FLAG_CHECK_FINITE, i.e.
    one launch per object, untuned) from the same state: the per-object copies
    take the batched parameters and Adam moments before each step, so that
    rounding-level differences, which Adam amplifies over many steps, do not
    accumulate between the two."""
    import torch

    objs = _setup()
    alt = _setup(seed=1)  # a second set of rays for the same objects
    stream = torch.cuda.Stream()
    ctx_b, ids_b = _make(pkg, objs, stream=stream)
    ctx_s, ids_s = _make(pkg, objs)
    opts = pkg.make_opts(nc=32, nr=32, lr=1e-2)
    opts_s = pkg.make_opts(nc=32, nr=32, lr=1e-2, flags=pkg.PRENOM_FLAG_CHECK_FINITE)
    loss_b = torch.zeros(len(objs), device="cuda")
    sets = [[_batch(o, i) for o, i in zip(src, ids_b)] for src in (objs, alt)]
    states = (pkg.PRENOM_STATE_THETA, pkg.PRENOM_STATE_ADAM_M, pkg.PRENOM_STATE_ADAM_V)
    torch.cuda.synchronize()
    for step in range(36):
        src = objs if step % 2 == 0 else alt
        if step > 0:
            for ib, i_s in zip(ids_b, ids_s):
                for w in states:
                    ctx_s.set_state(i_s, w, ctx_b.get_state(ib, w))
        with torch.cuda.stream(stream):
            ctx_b.train_step(sets[step % 2], opts, loss_b)
        stream.synchronize()
        lb = loss_b.cpu().numpy()
        for k, (o, i) in enumerate(zip(src, ids_s)):
            loss_s = torch.zeros(1, device="cuda")
            ctx_s.train_step([_batch(o, i)], opts_s, loss_s)
            assert abs(lb[k] - loss_s.item()) <= 1e-4 * abs(loss_s.item()) + 1e-7, (step, k)
        if step % 6 == 5:
            # Adam normalises each entry, so an entry whose gradient is at rounding level may
            # step either way (by at most lr): compare in bulk, and bound every entry by the step
            for k in range(len(objs)):
                tb = ctx_b.get_state(ids_b[k]).cpu().numpy()
                ts = ctx_s.get_state(ids_s[k]).cpu().numpy()
                close = np.abs(tb - ts) <= 1e-4 * np.abs(ts).max() + 1e-6
                assert np.mean(close) > 0.99, (step, k, np.mean(close))
                assert np.abs(tb - ts).max() <= 2 * 1e-2 * 1.01, (step, k)
    assert ctx_b.capture_count()[0] > 0  # the last steps replayed captured graphs
    assert "step " in ctx_b.tuning_report() and "=> " in ctx_b.tuning_report()  # the step-level choice was made
    for k in range(len(objs)):
        assert ctx_b.get_step(ids_b[k]) == 36 and ctx_s.get_step(ids_s[k]) == 36
    ctx_b.close()
    ctx_s.close()


def test_concurrent_groups_with_their_own_adam_passes(pkg):
    """PRENOM_FLAG_CONCURRENT: the step's groups (FP32, FP16 and BF16 objects of
    three widths) run concurrently on side streams, each followed by the Adam
    pass over its own objects, as a captured graph from the second step on.
    Every step against the same objects stepped one at a time from the same
    state (the per-object copies take the batched parameters and Adam moments
    before each step), with every object's step count advanced once."""
    import torch

    objs = _setup()
    stream = torch.cuda.Stream()
    ctx_b, ids_b = _make(pkg, objs, stream=stream)
    ctx_s, ids_s = _make(pkg, objs)
    flags = pkg.PRENOM_FLAG_SPLIT | pkg.PRENOM_FLAG_CONCURRENT  # untuned split form, no step-level trial
    opts = pkg.make_opts(nc=32, nr=32, lr=1e-2, flags=flags)
    opts_s = pkg.make_opts(nc=32, nr=32, lr=1e-2, flags=pkg.PRENOM_FLAG_CHECK_FINITE)
    loss_b = torch.zeros(len(objs), device="cuda")
    batches = [_batch(o, i) for o, i in zip(objs, ids_b)]
    states = (pkg.PRENOM_STATE_THETA, pkg.PRENOM_STATE_ADAM_M, pkg.PRENOM_STATE_ADAM_V)
    torch.cuda.synchronize()
    for step in range(4):
        if step > 0:
            for ib, i_s in zip(ids_b, ids_s):
                for w in states:
                    ctx_s.set_state(i_s, w, ctx_b.get_state(ib, w))
        with torch.cuda.stream(stream):
            ctx_b.train_step(batches, opts, loss_b)
        stream.synchronize()
        lb = loss_b.cpu().numpy()
        for k, (o, i) in enumerate(zip(objs, ids_s)):
            loss_s = torch.zeros(1, device="cuda")
            ctx_s.train_step([_batch(o, i)], opts_s, loss_s)
            assert abs(lb[k] - loss_s.item()) <= 1e-4 * abs(loss_s.item()) + 1e-7, (step, k)
            tb = ctx_b.get_state(ids_b[k]).cpu().numpy()
            ts = ctx_s.get_state(i).cpu().numpy()
            # Adam normalises each entry: an entry whose gradient is at rounding level may step
            # either way (by at most lr), so compare in bulk and bound every entry by the step
            close = np.abs(tb - ts) <= 1e-4 * np.abs(ts).max() + 1e-6
            assert np.mean(close) > 0.99, (step, k, np.mean(close))
            assert np.abs(tb - ts).max() <= 2 * 1e-2 * 1.01, (step, k)
    assert ctx_b.capture_count()[0] > 0  # replayed as a captured graph
    assert "step " not in ctx_b.tuning_report()  # no trial of one after the other against concurrently
    for k in range(len(objs)):
        assert ctx_b.get_step(ids_b[k]) == 4 and ctx_s.get_step(ids_s[k]) == 4
    ctx_b.close()
    ctx_s.close()


def test_mixed_precision_objects_of_a_batch_against_oracle(pkg):
    """The FP16 / BF16 objects of the mixed batch above against the oracle within
    the mixed-precision bounds (loss relative, gradient cosine and rel-L2)."""
    import torch

    # BF16 on the smallest networks of the table (L = 4 levels, one hidden layer of 16)
    # loses more: measured cos 0.99648, rel-L2 8.4e-2 on this batch's L=4 W=16 H=1 object
    # (the same in the split and the fused form; FP16 3.7e-3), frozen at cos >= 0.995,
    # rel-L2 <= 0.15 for BF16 here
    bounds = {1: dict(rel=5e-4, cos=0.99995, l2=1e-2), 2: dict(rel=5e-3, cos=0.995, l2=0.15)}
    objs = _setup(seed=3)
    ctx, ids = _make(pkg, objs)
    loss = torch.zeros(len(objs), device="cuda")
    ctx.train_step([_batch(o, i) for o, i in zip(objs, ids)], pkg.make_opts(nc=32, nr=32, flags=pkg.PRENOM_FLAG_NO_ADAM),
                   loss)
    for k, (o, i) in enumerate(zip(objs, ids)):
        if o["prec"] == 0:
            continue
        want = orc.batch(o["a"], o["theta"], o["grid"], o["rays"], 32, 32, t_in=o["t_in"], c_rand=o["cr"],
                         want_grad=True)
        g = ctx.get_state(i, pkg.PRENOM_STATE_GRAD).cpu().numpy().astype(np.float64)
        cos = float(g @ want["grad"] / (np.linalg.norm(g) * np.linalg.norm(want["grad"])))
        l2 = float(np.linalg.norm(g - want["grad"]) / np.linalg.norm(want["grad"]))
        b = bounds[o["prec"]]
        assert abs(loss[k].item() - want["loss"]) <= b["rel"] * abs(want["loss"]), k
        assert cos >= b["cos"] and l2 <= b["l2"], (k, cos, l2)
    ctx.close()


def test_stress_scale_batch_of_64_bf16_objects(pkg):
    """The mapping-stress configuration at test size: 64 objects of the category
    table (T 2^14..2^19, W 16/32/64, 1-3 hidden layers, L = 16, res 16..2048) in
    BF16, 64 samples per ray, one batched step; every object's loss against the
    oracle on identical samples within the BF16 bound, and the gradients of
    three objects (one per width)."""
    import torch
    from helpers import pool_cfg2
    from synth import init_params, prior_grid, random_colours, sample_batch, stratified_uniforms

    cats = [(17, 32, 1), (16, 32, 2), (19, 64, 3), (18, 64, 2), (14, 16, 1), (17, 32, 2), (14, 16, 1), (15, 16, 2),
            (19, 64, 3)]
    sc, pool = pool_cfg2()
    grid = prior_grid(sc, 64, 0)
    ctx = pkg.Context(seed=1)
    batches, host = [], []
    for i in range(64):
        log2T, W, H = cats[i % 9]
        a = orc.Arch(L=16, F=2, log2T=log2T, n_min=16, n_max=2048, width=W, hidden=H, lambda_d=0.1,
                     lambda_sigma=1e-3)
        theta = init_params(orc.n_hash_params(a), a.mlp_shapes(), 900 + i, hash_range=0.5).astype(np.float32)
        n = 16 + 8 * (i % 5)
        rays = sample_batch(pool, n, 400 + i)
        u = stratified_uniforms(n, 64, 500 + i)
        cr = random_colours(n, 600 + i)
        t_in = oracle_t(grid, rays, u, 64, 64)
        oid = ctx.create_object(pkg.make_arch(L=16, log2T=log2T, n_min=16, n_max=2048, width=W, hidden=H,
                                              lambda_d=0.1, lambda_sigma=1e-3, precision=2), theta)
        ctx.set_prior_grid(oid, grid)
        b = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in rays.items()}
        b.update(obj=oid, c_rand=torch.from_numpy(cr).cuda(), t_in=torch.from_numpy(t_in).cuda())
        batches.append(b)
        host.append((a, theta, rays, cr, t_in, oid, W))
    loss = torch.zeros(64, device="cuda")
    ctx.train_step(batches, pkg.make_opts(nc=64, nr=64, flags=pkg.PRENOM_FLAG_NO_ADAM), loss)
    lg = loss.cpu().numpy()
    checked = set()
    for k, (a, theta, rays, cr, t_in, oid, W) in enumerate(host):
        grad = W not in checked
        want = orc.batch(a, theta, grid, rays, 64, 64, t_in=t_in, c_rand=cr, want_grad=grad)
        assert abs(lg[k] - want["loss"]) <= 5e-3 * abs(want["loss"]), (k, lg[k], want["loss"])
        if grad:
            checked.add(W)
            g = ctx.get_state(oid, pkg.PRENOM_STATE_GRAD).cpu().numpy().astype(np.float64)
            cos = float(g @ want["grad"] / (np.linalg.norm(g) * np.linalg.norm(want["grad"])))
            l2 = float(np.linalg.norm(g - want["grad"]) / np.linalg.norm(want["grad"]))
            # one hidden layer of 16 in BF16 is the weakest network of the table (measured here
            # cos 0.99914, rel-L2 4.2e-2): the small-network BF16 bound of the test above
            c_min, l2_max = (0.995, 0.15) if W == 16 else (0.9995, 5e-2)
            assert cos >= c_min and l2 <= l2_max, (k, W, cos, l2)
    ctx.close()


def test_varying_ray_counts_bound_the_graph_cache(pkg):
    """70 steps with 70 different ray counts (70 step signatures, more than the
    64 graphs a context keeps) on a side stream: every step's loss follows the
    same object stepped without graphs or tuning (PRENOM_FLAG_CHECK_FINITE)."""
    import torch

    arch = dict(CFG1, log2T=14)
    a, theta, grid, rays, u, cr = case(arch, 400, 32, 32, seed=77, hash_range=0.5)
    o = dict(arch=arch, prec=0, a=a, theta=theta, grid=grid, rays=rays, cr=cr, t_in=oracle_t(grid, rays, u, 32, 32))
    stream = torch.cuda.Stream()
    ctx_g, (id_g,) = _make(pkg, [o], stream=stream)
    ctx_s, (id_s,) = _make(pkg, [o])
    opts = pkg.make_opts(nc=32, nr=32, lr=1e-2)
    opts_s = pkg.make_opts(nc=32, nr=32, lr=1e-2, flags=pkg.PRENOM_FLAG_CHECK_FINITE)
    full = _batch(o, id_g)
    full_s = _batch(o, id_s)
    lg, ls = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
    for step in range(70):
        n = 4 * (20 + step) - 1  # 4 rays per tile: 70 distinct tile counts, 70 step signatures
        with torch.cuda.stream(stream):
            ctx_g.train_step([{k: (v[:n] if torch.is_tensor(v) else v) for k, v in full.items()}], opts, lg)
        stream.synchronize()
        ctx_s.train_step([{k: (v[:n] if torch.is_tensor(v) else v) for k, v in full_s.items()}], opts_s, ls)
        assert abs(lg.item() - ls.item()) <= 1e-3 * abs(ls.item()), (step, lg.item(), ls.item())
    ctx_g.sync()
    ctx_g.close()
    ctx_s.close()
