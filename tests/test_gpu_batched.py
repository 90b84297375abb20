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
    """Twelve batched steps on a side stream: the first nine tune (one untimed
    call, then two rounds over the split form and three work-chunk sizes), the
    rest replay a captured graph while the ray buffers change; the losses and
    parameters follow the same objects stepped one at a time (with
    PRENOM_FLAG_CHECK_FINITE, i.e. one launch per object, untuned)."""
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
    torch.cuda.synchronize()
    for step in range(12):
        src = objs if step % 2 == 0 else alt
        with torch.cuda.stream(stream):
            ctx_b.train_step(sets[step % 2], opts, loss_b)
        stream.synchronize()
        lb = loss_b.cpu().numpy()
        for k, (o, i) in enumerate(zip(src, ids_s)):
            loss_s = torch.zeros(1, device="cuda")
            ctx_s.train_step([_batch(o, i)], opts_s, loss_s)
            assert abs(lb[k] - loss_s.item()) <= 1e-4 * abs(loss_s.item()) + 1e-7, (step, k)
    for k in range(len(objs)):
        assert ctx_b.get_step(ids_b[k]) == 12
        tb = ctx_b.get_state(ids_b[k]).cpu().numpy()
        ts = ctx_s.get_state(ids_s[k]).cpu().numpy()
        # Adam normalises each entry, so an entry whose gradient is at rounding level may step either
        # way (by at most lr per step): compare in bulk, and bound every entry by Adam's step size
        close = np.abs(tb - ts) <= 1e-4 * np.abs(ts).max() + 1e-6
        assert np.mean(close) > 0.99, (k, np.mean(close))
        assert np.abs(tb - ts).max() <= 2 * 1e-2 * 12 * 1.01, k
    ctx_b.close()
    ctx_s.close()
